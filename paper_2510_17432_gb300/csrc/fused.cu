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

#include <algorithm>
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

// ------------------------------------------------------------------ row-sweep two-step kernel
// One CTA owns a band of BX interior cells (plus one halo cell on each side: on the honeycomb the
// dependence of two steps reaches one cell, alternating A -> B(x-1) -> A(x-1)/A(x)) and a segment
// of SY rows, and sweeps the segment upwards.  Row r of phi_n streams into a ring of shared-memory
// rows with cp.async PD rows ahead; the step n+1 row r is formed from rows r-1, r, r+1 of phi_n
// and phi_{n-1}(r) (read straight into registers), kept in a three-row ring, and step n+2 row r-1
// follows from that ring.  Both new rows go to HBM once, so per two steps each state crosses HBM
// four times (plus the halo rows and columns) instead of six.  A tile row is CW = NT/P cells of
// 2 sites x P state pairs (contiguous in memory); thread t owns cell t/P, pair t%P, and both of
// its sites, so one of the three neighbours of each site is the thread's other site.  A shared row
// stores the A plane and the B plane of the tile separately (consecutive threads read consecutive
// 16-byte units, free of bank conflicts), each with P zero units before and after, which stand in
// for the neighbours outside the tile.
template <int NT_>
struct RowCfg {
  static constexpr int NT = NT_;
  static constexpr int RU = 2 * NT;      // thread units per tile row (two per thread)
  static constexpr int PD = 1;           // rows of phi_n in flight ahead of the one being waited for
  static constexpr int NSLOT0 = PD + 3;  // phi_n rows r-1 .. r+PD+1
  static constexpr int NSLOT1 = 3;       // phi_{n+1} rows r-2 .. r
  static constexpr int NV = 12;          // 2 steps x {A, Re B, Im B} x 2 states
  static constexpr int FOLD = 16;        // rows per FP32 partial (32 unit terms per thread)
  static constexpr int MINB = NT >= 256 ? 3 : 6;
  static size_t smem(int P) {
    return (size_t)(NSLOT0 + NSLOT1) * (RU + 4 * P) * 16 + (size_t)(NT / 32) * P * NV * 8;
  }
};

struct RowArgs {
  const float4* prev_in;  // phi_{n-1}
  const float4* cur_in;   // phi_n
  float4* prev_out;       // phi_{n+1}
  float4* cur_out;        // phi_{n+2}
  const float* diag;      // rescaled D_i or null
  float dc2, th2;
  int64_t Lx, Ly;
  int pbc_x, pbc_y;
  int P, logP, S;
  int CW, BX, SY;         // tile row cells, interior cells, rows per segment
  int nbx, nsy;           // bands, segments
  double* partials;       // [grid][P][NV]
  unsigned* counter;
  double* mu;
  int M;
  int step0;
};

__device__ __forceinline__ float4 f4lin(float d, float4 own, float th, float4 h, float4 pv) {
  return make_float4(d * own.x + th * h.x - pv.x, d * own.y + th * h.y - pv.y, d * own.z + th * h.z - pv.z,
                     d * own.w + th * h.w - pv.w);
}

template <int NT_, bool HAS_DIAG, bool OPEN>
__global__ void __launch_bounds__(NT_, RowCfg<NT_>::MINB) k_fused_rows(RowArgs a) {
  using RowC = RowCfg<NT_>;
  constexpr int NT = RowC::NT, RU = RowC::RU, NV = RowC::NV, NS0 = RowC::NSLOT0, NS1 = RowC::NSLOT1;
  extern __shared__ float4 smr[];
  __shared__ unsigned ticket;
  const int P = a.P, logP = a.logP, CW = a.CW, HALF = NT + 2 * P, RS = 2 * HALF;
  float4* ring0 = smr;                                  // [NS0][RS]
  float4* ring1 = smr + NS0 * RS;                       // [NS1][RS]
  double* red = reinterpret_cast<double*>(smr + (NS0 + NS1) * RS);  // [warps][P][NV]
  const int bx = blockIdx.x % a.nbx, sy = blockIdx.x / a.nbx;
  const int64_t x0 = (int64_t)bx * a.BX;                // first interior cell
  const int64_t ys = (int64_t)sy * a.SY;
  const int64_t ye = ys + a.SY < a.Ly ? ys + a.SY : a.Ly;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int i = threadIdx.x; i < (NS0 + NS1) * RS; i += NT) smr[i] = zero;
  for (int i = threadIdx.x; i < (NT / 32) * P * NV; i += NT) red[i] = 0.0;

  // this thread's cell c and pair p; a shared row holds the A units and then the B units of the
  // tile (each plane padded with P zero units on both sides), so a warp reads consecutive units
  const int c = threadIdx.x >> logP, p = threadIdx.x & (P - 1);
  const int wA = P + (int)threadIdx.x, wB = HALF + P + (int)threadIdx.x;
  int64_t x = x0 - 1 + c;
  bool ghx = false;
  if (x < 0 || x >= a.Lx) {
    if (OPEN && !a.pbc_x) ghx = true;
    else x = x < 0 ? x + a.Lx : (x >= a.Lx ? x - a.Lx : x);
    if (x < 0 || x >= a.Lx) ghx = true;  // a band wider than the lattice: never interior
  }
  const bool intx = c >= 1 && c <= CW - 2 && x0 + c - 1 < a.Lx;
  const int64_t colA = 2 * x * P + p;                  // unit offset of A(c) within a lattice row
  const int64_t row_units = 2 * a.Lx * P;
  auto grow = [&](int64_t r) -> int64_t {              // wrapped lattice row, or -1 for a ghost row
    if (r >= 0 && r < a.Ly) return r;
    if (OPEN && !a.pbc_y) return -1;
    return r < 0 ? r + a.Ly : r - a.Ly;
  };
  // ring slots: tile row ys-1+k lives in ring0 slot k % NS0 and ring1 slot k % NS1
  auto load_row = [&](int64_t r, int slot) {  // phi_n row r (zero for ghosts / rows past the end)
    const int64_t gy = (r <= ye) ? grow(r) : -1;
    float4* dst = ring0 + slot * RS;
    const bool ok = gy >= 0 && !ghx;
    const float4* src = ok ? a.cur_in + gy * row_units + colA : a.cur_in;
    cp_async16(dst + wA, src, ok ? 16 : 0);
    cp_async16(dst + wB, ok ? src + P : a.cur_in, ok ? 16 : 0);
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  auto diag2 = [&](int64_t gy) -> float2 {             // 2 D of A(c) and B(c) in row gy
    if (!HAS_DIAG) return make_float2(a.dc2, a.dc2);
    if (gy < 0 || ghx) return make_float2(0.f, 0.f);
    const float2 d = __ldg(reinterpret_cast<const float2*>(a.diag + 2 * (gy * a.Lx + x)));
    return make_float2(2.f * d.x, 2.f * d.y);
  };

  float acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0.f;
  int folded = 0;
  // every FOLD rows: each thread's FP32 partials (32 unit terms) are summed over the lanes of its
  // pair by a fixed FP32 tree and added in FP64 to the warp's slot
  auto fold = [&]() {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      float t = acc[v];
      for (int off = 16; off >= P; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
      if (lane < P) red[(warp * P + lane) * NV + v] += (double)t;
      acc[v] = 0.f;
    }
  };
  auto moments = [&](int base, float4 own, float4 o) {  // FFMA chains into the FP32 partials
    acc[base + 0] = fmaf(own.x, own.x, fmaf(own.y, own.y, acc[base + 0]));
    acc[base + 1] = fmaf(o.x, own.x, fmaf(o.y, own.y, acc[base + 1]));
    acc[base + 2] = fmaf(o.x, own.y, fmaf(-o.y, own.x, acc[base + 2]));
    acc[base + 3] = fmaf(own.z, own.z, fmaf(own.w, own.w, acc[base + 3]));
    acc[base + 4] = fmaf(o.z, own.z, fmaf(o.w, own.w, acc[base + 4]));
    acc[base + 5] = fmaf(o.z, own.w, fmaf(-o.w, own.z, acc[base + 5]));
  };

  const float th = a.th2;
  // prologue: rows ys-1 .. ys-1+PD (the first iteration reads r-1 .. r+1 = ys-2 .. ys; row ys-2 only
  // feeds A sites of the halo row ys-1, which no interior value uses, and its slot holds zeros)
  for (int k = 0; k <= RowC::PD; ++k) load_row(ys - 1 + k, k);
  float4 pvA, pvB;  // phi_{n-1} of the row being advanced
  {
    const int64_t gy = grow(ys - 1);
    const bool ok = gy >= 0 && !ghx;
    pvA = ok ? __ldcs(a.prev_in + gy * row_units + colA) : zero;
    pvB = ok ? __ldcs(a.prev_in + gy * row_units + colA + P) : zero;
  }
  float2 dPrev = make_float2(0.f, 0.f);  // 2 D of the row below (step n+2 runs one row behind)
  int k0 = 0, k1 = 0;                    // ring0 / ring1 slots of row r
  for (int64_t r = ys - 1; r <= ye; ++r) {
    // rows up to r+1 complete; rows r+2 .. r+PD may still be in flight
    asm volatile("cp.async.wait_group %0;" ::"n"(RowC::PD - 1) : "memory");
    __syncthreads();
    const int km1 = k0 == 0 ? NS0 - 1 : k0 - 1;   // row r-1
    const int kp1 = k0 == NS0 - 1 ? 0 : k0 + 1;   // row r+1
    const int km2 = km1 == 0 ? NS0 - 1 : km1 - 1; // row r-2 = row r+PD+1 (NS0 = PD+3)
    load_row(r + RowC::PD + 1, km2);              // the previous iteration used row r-2 last
    const float4* Rm = ring0 + km1 * RS;
    const float4* R0 = ring0 + k0 * RS;
    const float4* Rp = ring0 + kp1 * RS;
    float4* Q0 = ring1 + k1 * RS;
    const int64_t gy = grow(r);
    const bool ghost = gy < 0 || ghx;
    // ---- step n+1 at row r: A(c) <- B(c), B(c-1), B(c, r-1);  B(c) <- A(c), A(c+1), A(c, r+1)
    {
      const float4 a0 = R0[wA], b0 = R0[wB];
      const float4 hA = f4add(f4add(b0, R0[wB - P]), Rm[wB]);
      const float4 hB = f4add(f4add(a0, R0[wA + P]), Rp[wA]);
      const float2 d = diag2(gy);
      float4 oA = f4lin(d.x, a0, th, hA, pvA);
      float4 oB = f4lin(d.y, b0, th, hB, pvB);
      if (OPEN && ghost) {
        oA = zero;
        oB = zero;
      }
      Q0[wA] = oA;
      Q0[wB] = oB;
      if (r >= ys && r < ye && intx) {
        const int64_t u = gy * row_units + colA;
        __stcs(a.prev_out + u, oA);
        __stcs(a.prev_out + u + P, oB);
        moments(0, a0, oA);
        moments(0, b0, oB);
      }
      // phi_{n-1} of the next row, in flight during the second step
      const int64_t gn = (r + 1 <= ye) ? grow(r + 1) : -1;
      const bool okn = gn >= 0 && !ghx;
      pvA = okn ? __ldcs(a.prev_in + gn * row_units + colA) : zero;
      pvB = okn ? __ldcs(a.prev_in + gn * row_units + colA + P) : zero;
      const float2 dq = dPrev;
      dPrev = d;
      __syncthreads();
      // ---- step n+2 at row q = r-1 from phi_{n+1} rows q-1, q, q+1 = r and phi_n(q)
      const int64_t q = r - 1;
      if (q >= ys && q < ye && intx) {
        const float4* Qc = ring1 + (k1 == 0 ? 2 : k1 - 1) * RS;  // row r-1
        const float4* Qm = ring1 + (k1 == 2 ? 0 : k1 + 1) * RS;  // row r-2
        const float4 a1 = Qc[wA], b1 = Qc[wB];
        const float4 gA = f4add(f4add(b1, Qc[wB - P]), Qm[wB]);
        const float4 gB = f4add(f4add(a1, Qc[wA + P]), Q0[wA]);
        const float4 nA = f4lin(dq.x, a1, th, gA, Rm[wA]);
        const float4 nB = f4lin(dq.y, b1, th, gB, Rm[wB]);
        const int64_t u = grow(q) * row_units + colA;
        __stcs(a.cur_out + u, nA);
        __stcs(a.cur_out + u + P, nB);
        moments(6, a1, nA);
        moments(6, b1, nB);
      }
    }
    if (++folded == RowC::FOLD) {
      folded = 0;
      fold();
    }
    k0 = kp1;
    k1 = k1 == 2 ? 0 : k1 + 1;
  }
  fold();
  __syncthreads();
  // per-CTA partials [P][NV] (warps in order), then the last CTA sums them in CTA order
  for (int q = threadIdx.x; q < P * NV; q += NT) {
    const int pp = q / NV, v = q - pp * NV;
    double t = 0.0;
    for (int w = 0; w < NT / 32; ++w) t += red[(w * P + pp) * NV + v];
    a.partials[(size_t)blockIdx.x * P * NV + q] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(a.counter, 1u);
  __syncthreads();
  if (ticket != gridDim.x - 1) return;
  __threadfence();
  const int nval = 2 * a.S * 3;
  for (int v = warp; v < nval; v += NT / 32) {
    const int k = v / (a.S * 3), rem = v - k * a.S * 3, s = rem / 3, comp = rem - s * 3;
    const int pr = s >> 1, sub = s & 1;
    const int idx = k * 6 + sub * 3 + comp;
    double sum = 0.0;
    for (int t = lane; t < (int)gridDim.x; t += 32) sum += __ldcg(a.partials + ((size_t)t * P + pr) * NV + idx);
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

// ------------------------------------------------------------------ row sweep, K steps per pass
// The same sweep with K (even) levels: at tile row r level L forms phi_{n+L} at row r - (L-1) from
// level L-1's ring (rows r-L .. r-L+2) and phi_{n+L-2} at that row (level L-2's ring, phi_n's ring
// for L = 2, registers for L = 1).  Levels 1 .. K-1 keep three-row rings; levels K-1 and K go to
// HBM.  The exact region shrinks by one cell / row per two steps, so the tile carries K/2 halo
// cells on each side and the segment K/2 halo rows below and above.
template <int NT_, int K_>
struct RowKCfg {
  static constexpr int NT = NT_, K = K_, H = K_ / 2;
  static constexpr int RU = 2 * NT;
  static constexpr int PD = 1;
  static constexpr int NSLOT0 = PD + 3;
  static constexpr int NV = 6 * K;
  static constexpr int FOLD = 16;
  static constexpr int MINB = K == 2 ? (NT >= 256 ? 3 : 6) : (NT >= 256 ? 2 : 4);
  // rows: [P zero][A plane: NT units][P zero][B plane: NT units][P zero]; the middle pad serves
  // both A(c+1) past the last cell and B(c-1) before the first
  static size_t smem(int P) {
    return (size_t)(NSLOT0 + 3 * (K - 1)) * (RU + 3 * P) * 16 + (size_t)(NT / 32) * P * NV * 8;
  }
};

template <int NT_, int K_, bool HAS_DIAG, bool OPEN>
__global__ void __launch_bounds__(NT_, RowKCfg<NT_, K_>::MINB) k_fused_rowsK(RowArgs a) {
  using RC = RowKCfg<NT_, K_>;
  constexpr int NT = RC::NT, K = RC::K, H = RC::H, RU = RC::RU, NV = RC::NV, NS0 = RC::NSLOT0;
  extern __shared__ float4 smr[];
  __shared__ unsigned ticket;
  const int P = a.P, logP = a.logP, CW = a.CW, RS = 2 * NT + 3 * P;
  float4* ring0 = smr;                                   // [NS0][RS]
  float4* ringL = smr + NS0 * RS;                        // [K-1][3][RS]: level L at ringL + (L-1)*3*RS
  double* red = reinterpret_cast<double*>(smr + (NS0 + 3 * (K - 1)) * RS);  // [warps][P][NV]
  const int bx = blockIdx.x % a.nbx, sy = blockIdx.x / a.nbx;
  const int64_t x0 = (int64_t)bx * a.BX;
  const int64_t ys = (int64_t)sy * a.SY;
  const int64_t ye = ys + a.SY < a.Ly ? ys + a.SY : a.Ly;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int i = threadIdx.x; i < (NS0 + 3 * (K - 1)) * RS; i += NT) smr[i] = zero;
  for (int i = threadIdx.x; i < (NT / 32) * P * NV; i += NT) red[i] = 0.0;

  const int c = threadIdx.x >> logP, p = threadIdx.x & (P - 1);
  const int wA = P + (int)threadIdx.x, wB = NT + 2 * P + (int)threadIdx.x;
  int64_t x = x0 - H + c;
  bool ghx = false;
  if (x < 0 || x >= a.Lx) {
    if (OPEN && !a.pbc_x) ghx = true;
    else x = x < 0 ? x + a.Lx : (x >= a.Lx ? x - a.Lx : x);
    if (x < 0 || x >= a.Lx) ghx = true;
  }
  const bool intx = c >= H && c < CW - H && x0 + c - H < a.Lx;
  const int64_t colA = 2 * x * P + p;
  const int64_t row_units = 2 * a.Lx * P;
  const int64_t r0 = ys - H;                  // first tile row; tile row r0+k: ring0 slot k % NS0, ring slot k % 3
  const int64_t rlast_load = ye + H - 1;      // last phi_n row that any exact value needs
  auto grow = [&](int64_t r) -> int64_t {
    if (r >= 0 && r < a.Ly) return r;
    if (OPEN && !a.pbc_y) return -1;
    return r < 0 ? r + a.Ly : r - a.Ly;
  };
  auto load_row = [&](int64_t r, int slot) {
    const int64_t gy = (r <= rlast_load) ? grow(r) : -1;
    float4* dst = ring0 + slot * RS;
    const bool ok = gy >= 0 && !ghx;
    const float4* src = ok ? a.cur_in + gy * row_units + colA : a.cur_in;
    cp_async16(dst + wA, src, ok ? 16 : 0);
    cp_async16(dst + wB, ok ? src + P : a.cur_in, ok ? 16 : 0);
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  auto diag2 = [&](int64_t gy) -> float2 {
    if (!HAS_DIAG) return make_float2(a.dc2, a.dc2);
    if (gy < 0 || ghx) return make_float2(0.f, 0.f);
    const float2 d = __ldg(reinterpret_cast<const float2*>(a.diag + 2 * (gy * a.Lx + x)));
    return make_float2(2.f * d.x, 2.f * d.y);
  };
  float acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0.f;
  int folded = 0;
  // every FOLD rows: FP32 lane tree per pair, added in FP64 to the warp's slots
  auto fold = [&]() {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      float t = acc[v];
      for (int off = 16; off >= P; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
      if (lane < P) red[(warp * P + lane) * NV + v] += (double)t;
      acc[v] = 0.f;
    }
  };
  auto moments = [&](int base, float4 own, float4 o) {
    acc[base + 0] = fmaf(own.x, own.x, fmaf(own.y, own.y, acc[base + 0]));
    acc[base + 1] = fmaf(o.x, own.x, fmaf(o.y, own.y, acc[base + 1]));
    acc[base + 2] = fmaf(o.x, own.y, fmaf(-o.y, own.x, acc[base + 2]));
    acc[base + 3] = fmaf(own.z, own.z, fmaf(own.w, own.w, acc[base + 3]));
    acc[base + 4] = fmaf(o.z, own.z, fmaf(o.w, own.w, acc[base + 4]));
    acc[base + 5] = fmaf(o.z, own.w, fmaf(-o.w, own.z, acc[base + 5]));
  };

  const float th = a.th2;
  for (int k = 0; k <= RC::PD; ++k) load_row(r0 + k, k);
  float4 pvA, pvB;
  {
    const int64_t gy = grow(r0);
    const bool ok = gy >= 0 && !ghx && r0 <= rlast_load;
    pvA = ok ? __ldcs(a.prev_in + gy * row_units + colA) : zero;
    pvB = ok ? __ldcs(a.prev_in + gy * row_units + colA + P) : zero;
  }
  float2 dRow[K];  // 2 D of rows r, r-1, .., r-K+1
#pragma unroll
  for (int l = 0; l < K; ++l) dRow[l] = make_float2(0.f, 0.f);
  int k0 = 0, k1 = 0;  // ring0 / level-ring slots of row r
  const int64_t r_end = ye + K - 2;
  for (int64_t r = r0; r <= r_end; ++r) {
    asm volatile("cp.async.wait_group %0;" ::"n"(RC::PD - 1) : "memory");
    __syncthreads();
    const int km1 = k0 == 0 ? NS0 - 1 : k0 - 1;
    const int kp1 = k0 == NS0 - 1 ? 0 : k0 + 1;
    const int km2 = km1 == 0 ? NS0 - 1 : km1 - 1;
    load_row(r + RC::PD + 1, km2);
#pragma unroll
    for (int l = K - 1; l > 0; --l) dRow[l] = dRow[l - 1];
    dRow[0] = diag2(grow(r));
    // ring slot (0..2) of row r - j
    auto rs = [&](int j) -> int { return (k1 - j + 6) % 3; };
#pragma unroll
    for (int L = 1; L <= K; ++L) {
      const int64_t q = r - (L - 1);
      const int64_t gq = grow(q);
      const bool ghost = gq < 0 || ghx;
      float4 own_a, own_b, nA, nB;
      if (L == 1) {
        const float4* Rm = ring0 + km1 * RS;
        const float4* R0 = ring0 + k0 * RS;
        const float4* Rp = ring0 + kp1 * RS;
        own_a = R0[wA];
        own_b = R0[wB];
        const float4 hA = f4add(f4add(own_b, R0[wB - P]), Rm[wB]);
        const float4 hB = f4add(f4add(own_a, R0[wA + P]), Rp[wA]);
        nA = f4lin(dRow[0].x, own_a, th, hA, pvA);
        nB = f4lin(dRow[0].y, own_b, th, hB, pvB);
      } else {
        const float4* In = ringL + (L - 2) * 3 * RS;      // level L-1
        const float4* Qm = In + rs(L) * RS;               // row q-1 = r-L
        const float4* Qc = In + rs(L - 1) * RS;           // row q
        const float4* Qp = In + rs(L - 2) * RS;           // row q+1
        const float4* Pv = (L == 2) ? ring0 + km1 * RS : ringL + (L - 3) * 3 * RS + rs(L - 1) * RS;
        own_a = Qc[wA];
        own_b = Qc[wB];
        const float4 gA = f4add(f4add(own_b, Qc[wB - P]), Qm[wB]);
        const float4 gB = f4add(f4add(own_a, Qc[wA + P]), Qp[wA]);
        nA = f4lin(dRow[L - 1].x, own_a, th, gA, Pv[wA]);
        nB = f4lin(dRow[L - 1].y, own_b, th, gB, Pv[wB]);
      }
      if (OPEN && ghost) {
        nA = zero;
        nB = zero;
      }
      if (L < K) {
        float4* Out = ringL + (L - 1) * 3 * RS + rs(L - 1) * RS;
        Out[wA] = nA;
        Out[wB] = nB;
      }
      const bool inside = q >= ys && q < ye && intx;
      if (inside) {
        if (L >= K - 1) {
          float4* dst = (L == K - 1) ? a.prev_out : a.cur_out;
          const int64_t u = gq * row_units + colA;
          __stcs(dst + u, nA);
          __stcs(dst + u + P, nB);
        }
        moments((L - 1) * 6, own_a, nA);
        moments((L - 1) * 6, own_b, nB);
      }
      if (L == 1) {  // phi_{n-1} of the next row, in flight during the later levels
        const int64_t gn = (r + 1 <= rlast_load) ? grow(r + 1) : -1;
        const bool okn = gn >= 0 && !ghx;
        pvA = okn ? __ldcs(a.prev_in + gn * row_units + colA) : zero;
        pvB = okn ? __ldcs(a.prev_in + gn * row_units + colA + P) : zero;
      }
      if (L < K) __syncthreads();
    }
    if (++folded == RC::FOLD) {
      folded = 0;
      fold();
    }
    k0 = kp1;
    k1 = k1 == 2 ? 0 : k1 + 1;
  }
  fold();
  __syncthreads();
  for (int q = threadIdx.x; q < P * NV; q += NT) {  // warps in order
    const int pp = q / NV, v = q - pp * NV;
    double t = 0.0;
    for (int w = 0; w < NT / 32; ++w) t += red[(w * P + pp) * NV + v];
    a.partials[(size_t)blockIdx.x * P * NV + q] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(a.counter, 1u);
  __syncthreads();
  if (ticket != gridDim.x - 1) return;
  __threadfence();
  const int nval = K * a.S * 3;
  for (int v = warp; v < nval; v += NT / 32) {
    const int k = v / (a.S * 3), rem = v - k * a.S * 3, s = rem / 3, comp = rem - s * 3;
    const int pr = s >> 1, sub = s & 1;
    const int idx = k * 6 + sub * 3 + comp;
    double sum = 0.0;
    for (int t = lane; t < (int)gridDim.x; t += 32) sum += __ldcg(a.partials + ((size_t)t * P + pr) * NV + idx);
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

template <int NT, bool D, bool O>
static cudaError_t set_rows_smem() {
  return cudaFuncSetAttribute(fused::k_fused_rows<NT, D, O>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)fused::RowCfg<NT>::smem(16));
}

template <int NT>
static int launch_rows(tbpm_ctx* ctx, const tbpm_lattice* lat, const RecurrenceArgs& ra, const void* prev_in,
                       const void* cur_in, void* prev_out, void* cur_out, int step0) {
  using namespace fused;
  using RowC = RowCfg<NT>;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    cudaError_t e[4] = {set_rows_smem<NT, false, false>(), set_rows_smem<NT, false, true>(),
                        set_rows_smem<NT, true, false>(), set_rows_smem<NT, true, true>()};
    for (cudaError_t x : e)
      if (x != cudaSuccess) attr = x;
  });
  TBPM_CK(attr);
  RowArgs a;
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
  a.logP = 0;
  while ((1 << a.logP) < a.P) ++a.logP;
  a.S = ra.S;
  a.CW = RowC::RU / (2 * a.P);
  a.BX = a.CW - 2;
  a.nbx = (int)((a.Lx + a.BX - 1) / a.BX);
  // one wave: as many row segments as leave every resident CTA slot busy once (long segments also
  // keep the halo-row overhead, 2 rows per segment, small)
  static int per_sm = 0;
  if (per_sm == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused_rows<NT, false, false>, NT,
                                                      RowC::smem(a.P)) != cudaSuccess || per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
  }
  // segments per band: the count whose CTAs fill the resident slots best over whole waves, weighed
  // by what each segment adds (one wave when it fits, e.g. 2048 x 2048)
  const int64_t slots = (int64_t)ctx->num_sms * per_sm;
  const int64_t max_nsy = std::max<int64_t>(1, std::min<int64_t>(a.Ly / 4, 8 * slots / a.nbx + 1));
  int64_t nsy = 1;
  double best = -1.0;
  for (int64_t k = 1; k <= max_nsy; ++k) {
    const int64_t sy = (a.Ly + k - 1) / k;
    const int64_t ctas = a.nbx * ((a.Ly + sy - 1) / sy);
    const int64_t waves = (ctas + slots - 1) / slots;
    // a segment costs its two halo rows plus the fill and drain of the row pipeline (~6 rows)
    const double eff = (double)ctas / (double)(waves * slots) * (double)sy / (double)(sy + 8);
    if (eff > best + 1e-9) {
      best = eff;
      nsy = k;
    }
  }
  a.SY = (int)((a.Ly + nsy - 1) / nsy);
  a.nsy = (int)((a.Ly + a.SY - 1) / a.SY);
  a.mu = ra.mu;
  a.M = ra.M;
  a.step0 = step0;
  const int64_t grid = (int64_t)a.nbx * a.nsy;
  TBPM_TRY(ensure(ctx, ctx->ws_fused_partials, sizeof(double) * RowC::NV * (size_t)a.P * (size_t)grid));
  a.partials = (double*)ctx->ws_fused_partials.p;
  a.counter = ra.counter;
  const bool open = !(a.pbc_x && a.pbc_y);
  const dim3 gr((unsigned)grid), bl(NT);
  const size_t sm = RowC::smem(a.P);
  if (a.diag) {
    if (open) k_fused_rows<NT, true, true><<<gr, bl, sm, ctx->stream>>>(a);
    else k_fused_rows<NT, true, false><<<gr, bl, sm, ctx->stream>>>(a);
  } else {
    if (open) k_fused_rows<NT, false, true><<<gr, bl, sm, ctx->stream>>>(a);
    else k_fused_rows<NT, false, false><<<gr, bl, sm, ctx->stream>>>(a);
  }
  TBPM_CK_LAUNCH(ctx);
  return TBPM_OK;
}

template <int NT, int K, bool D, bool O>
static cudaError_t set_rowsK_smem() {
  return cudaFuncSetAttribute(fused::k_fused_rowsK<NT, K, D, O>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)fused::RowKCfg<NT, K>::smem(16));
}

template <int NT, int K>
static int launch_rowsK(tbpm_ctx* ctx, const tbpm_lattice* lat, const RecurrenceArgs& ra, const void* prev_in,
                        const void* cur_in, void* prev_out, void* cur_out, int step0) {
  using namespace fused;
  using RC = RowKCfg<NT, K>;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    cudaError_t e[4] = {set_rowsK_smem<NT, K, false, false>(), set_rowsK_smem<NT, K, false, true>(),
                        set_rowsK_smem<NT, K, true, false>(), set_rowsK_smem<NT, K, true, true>()};
    for (cudaError_t x : e)
      if (x != cudaSuccess) attr = x;
  });
  TBPM_CK(attr);
  RowArgs a;
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
  a.logP = 0;
  while ((1 << a.logP) < a.P) ++a.logP;
  a.S = ra.S;
  a.CW = RC::RU / (2 * a.P);
  a.BX = a.CW - 2 * RC::H;
  if (a.BX < 1) {
    set_error("fused pass: tile too narrow for %d states", a.S);
    return TBPM_EUNSUPPORTED;
  }
  a.nbx = (int)((a.Lx + a.BX - 1) / a.BX);
  static int per_sm = 0;
  if (per_sm == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused_rowsK<NT, K, false, false>, NT,
                                                      RC::smem(a.P)) != cudaSuccess || per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
  }
  const int64_t slots = (int64_t)ctx->num_sms * per_sm;
  const int64_t max_nsy = std::max<int64_t>(1, std::min<int64_t>(a.Ly / 4, 8 * slots / a.nbx + 1));
  int64_t nsy = 1;
  double best = -1.0;
  for (int64_t k = 1; k <= max_nsy; ++k) {
    const int64_t sy = (a.Ly + k - 1) / k;
    const int64_t ctas = a.nbx * ((a.Ly + sy - 1) / sy);
    const int64_t waves = (ctas + slots - 1) / slots;
    const double eff = (double)ctas / (double)(waves * slots) * (double)sy / (double)(sy + K + 6);
    if (eff > best + 1e-9) {
      best = eff;
      nsy = k;
    }
  }
  a.SY = (int)((a.Ly + nsy - 1) / nsy);
  a.nsy = (int)((a.Ly + a.SY - 1) / a.SY);
  a.mu = ra.mu;
  a.M = ra.M;
  a.step0 = step0;
  const int64_t grid = (int64_t)a.nbx * a.nsy;
  TBPM_TRY(ensure(ctx, ctx->ws_fused_partials, sizeof(double) * RC::NV * (size_t)a.P * (size_t)grid));
  a.partials = (double*)ctx->ws_fused_partials.p;
  a.counter = ra.counter;
  const bool open = !(a.pbc_x && a.pbc_y);
  const dim3 gr((unsigned)grid), bl(NT);
  const size_t sm = RC::smem(a.P);
  if (a.diag) {
    if (open) k_fused_rowsK<NT, K, true, true><<<gr, bl, sm, ctx->stream>>>(a);
    else k_fused_rowsK<NT, K, true, false><<<gr, bl, sm, ctx->stream>>>(a);
  } else {
    if (open) k_fused_rowsK<NT, K, false, true><<<gr, bl, sm, ctx->stream>>>(a);
    else k_fused_rowsK<NT, K, false, false><<<gr, bl, sm, ctx->stream>>>(a);
  }
  TBPM_CK_LAUNCH(ctx);
  return TBPM_OK;
}

bool fused_applicable(const tbpm_lattice* lat, int precision, int Spad) {
  const Geom& g = lat->geom;
  return lat->path == TBPM_PATH_STENCIL && g.kind == TBPM_HONEYCOMB && precision == TBPM_C64 && Spad >= 2 &&
         g.Lx >= fused::V1::WX && g.Ly >= fused::V1::WY;
}

int fused_steps(int variant) { return (variant == 1 || (variant >= 5 && variant != 7)) ? 4 : 2; }

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
  if (variant >= 8 && variant <= 10) {
    // the register sweep copies whole band rows; a lattice narrower than a band takes mode 5
    const int band = (variant == 8 ? 128 : variant == 9 ? 192 : 256) / (ra.S / 2);
    if (lat->geom.Lx >= band)
      return launch_sweep_pass(ctx, lat, ra, prev_in, cur_in, prev_out, cur_out, step0, variant);
    variant = 5;
  }
  if (variant == 5) return launch_rowsK<128, 4>(ctx, lat, ra, prev_in, cur_in, prev_out, cur_out, step0);
  if (variant == 6) return launch_rowsK<256, 4>(ctx, lat, ra, prev_in, cur_in, prev_out, cur_out, step0);
  if (variant == 7) return launch_rowsK<256, 2>(ctx, lat, ra, prev_in, cur_in, prev_out, cur_out, step0);
  if (variant == 3) return launch_rows<128>(ctx, lat, ra, prev_in, cur_in, prev_out, cur_out, step0);
  if (variant == 4) return launch_rows<256>(ctx, lat, ra, prev_in, cur_in, prev_out, cur_out, step0);
  if (variant == 2) return launch_variant<fused::V2>(ctx, lat, ra, prev_in, cur_in, prev_out, cur_out, step0);
  return launch_variant<fused::V1>(ctx, lat, ra, prev_in, cur_in, prev_out, cur_out, step0);
}

}  // namespace tbpm
