// Register-resident row sweep: K Chebyshev steps per pass over HBM on the honeycomb stencil,
// complex64 state pairs, with the moment inner products of every step fused in.
//
// The recurrence phi_{n+1} = 2 H~ phi_n - phi_{n-1} (App. B) on the honeycomb couples
//   A(x,y) <- B(x,y), B(x-1,y), B(x,y-1)        B(x,y) <- A(x,y), A(x+1,y), A(x,y+1)
// so a thread that owns one cell (both sites) and one state pair finds every neighbour in its
// own registers except B(x-1,y) and A(x+1,y), which belong to the threads of the adjacent cells
// of the same row.  A CTA owns a band of CW cells (K/2 halo cells on each side) and a segment of
// rows (K/2 halo rows below and above) and sweeps it upwards as a wavefront: at sweep position r
// level L = 1..K forms phi_{n+L} at row r - (L-1) from
//   * level L-1 at rows r-L, r-L+1, r-L+2 of the same cell: registers (the thread formed them in
//     this and the two previous positions),
//   * level L-1 at row r-L+1 of the adjacent cells: a shared-memory exchange row written in the
//     previous position (double-buffered, so one barrier per position suffices),
//   * level L-2 at row r-L+1 of the same cell: registers.
// Level 0 (phi_n) and phi_{n-1} arrive row by row through 1-D TMA bulk copies (cp.async.bulk,
// one elected thread, an mbarrier per ring slot) into a ring NSLOT rows deep; a band row is
// contiguous in the [N][S] layout, so one copy per state block (two where a periodic band wraps).
// Levels K-1 and K go to HBM, so per K steps each state block crosses HBM four times: read
// phi_{n-1}, phi_n, write phi_{n+K-1}, phi_{n+K}.
//
// Moments (cost halving of Eq. cheby_prod): for every level, <phi_{n+L-1}|phi_{n+L-1}> and
// <phi_{n+L}|phi_{n+L-1}> over the segment's interior, summed in FP32 over at most 32 units per
// thread, then FP32 lane trees per state pair, FP64 warp slots, FP64 block partials and a
// fixed-order FP64 sum by the last CTA: deterministic for a given launch shape.
//
// Every mbarrier wait is bounded by a wall-clock budget; on expiry the CTA records an error code
// in the caller's status word, stops sweeping, waits (bounded) for its copies in flight and still
// takes part in the grid reduction so that the completion counter stays consistent.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "tbpm_internal.cuh"

namespace tbpm {
namespace sweep {

constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s per mbarrier wait

// Source of the bulk copies for rows that hold no data (outside an open lattice, beyond the rows
// a segment needs): two state-block rows of 2 NT units for NT <= 256.  Zero-initialised when the
// module loads and never written, so every ring read is a plain shared load.
static __device__ __align__(16) float4 g_zero_rows[2 * 256];

template <int NT_, int K_, int NSLOT_>
struct Cfg {
  static constexpr int NT = NT_, K = K_, H = K_ / 2, NSLOT = NSLOT_;
  static constexpr int NV = 4 * K;     // per level: {|a|^2, Re<n|a>} x 2 states
  static constexpr int FOLD = 16;      // positions per FP32 partial (32 unit terms per thread)
  static constexpr int MINB = NT <= 128 ? 3 : NT <= 192 ? 2 : 1;
  static constexpr int BAR_BYTES = ((NSLOT * 8 + 15) / 16) * 16;
  // ring slot: [P zero][phi_n row: 2 NT units][P zero][phi_{n-1} row: 2 NT units], padded to a
  // multiple of 8 units (128 bytes) so that every slot starts on the same bank
  __host__ __device__ static int slot_units(int P) { return (4 * NT + 2 * P + 7) & ~7; }
  // exchange row: [A plane: NT units][P zero][B plane: NT units]
  __host__ __device__ static int xrow_units(int P) { return 2 * NT + P; }
  // + disordered lattices: a thread-private ring of 2 D for the last 4 rows ([4][NT] float2)
  static size_t smem(int P, bool diag) {
    return (size_t)BAR_BYTES + 16 * ((size_t)NSLOT * slot_units(P) + (size_t)2 * (K - 1) * xrow_units(P)) +
           8 * (size_t)(NT / 32) * P * NV + (diag ? (size_t)8 * 4 * NT : 0);
  }
};

struct Args {
  const float4* prev_in;  // phi_{n-1}
  const float4* cur_in;   // phi_n
  float4* prev_out;       // phi_{n+K-1}
  float4* cur_out;        // phi_{n+K}
  const float* diag;      // rescaled D_i or null
  float dc2, th2;         // 2 D (clean lattice), 2 t/|H|
  int64_t Lx, Ly;
  int pbc_x, pbc_y;
  int P, logP, S;
  int CW, BX, SY;         // band cells, interior cells, rows per segment
  int nbx, nsy;
  double* partials;       // [grid][P][NV]
  unsigned* counter;
  double* mu;
  int M;
  int step0;
  int* status;            // host-visible status word: nonzero = a bounded wait expired
  float4* win[4];         // window mode: phi_{n+1} .. phi_{n+4}, one buffer each
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// Bounded wait for the phase of the given parity: false once budget_ns of wall-clock time has
// passed without the phase completing.
__device__ __forceinline__ bool mbar_wait_ns(uint32_t bar, uint32_t parity, uint64_t budget_ns) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (!mbar_try(bar, parity))
    if (globaltimer() - t0 > budget_ns) return false;
  return true;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  return mbar_wait_ns(bar, parity, kWaitNs);
}

// 1-D bulk copy global -> shared, completion counted in bytes on the mbarrier.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// d own + th (n1 + n2 + n3) - pv for one complex64 pair, as two packed f32x2 halves (one state each)
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 half_update(float2 d, float2 own, float2 th, float2 n1, float2 n2, float2 n3,
                                              float2 pv) {
  const float2 h = __fadd2_rn(__fadd2_rn(n1, n2), n3);
  return __ffma2_rn(d, own, __ffma2_rn(th, h, make_float2(-pv.x, -pv.y)));
}
__device__ __forceinline__ float4 level_update(float d, float4 own, float th, float4 n1, float4 n2, float4 n3,
                                               float4 pv) {
  const float2 d2 = make_float2(d, d), t2 = make_float2(th, th);
  const float2 l = half_update(d2, lo2(own), t2, lo2(n1), lo2(n2), lo2(n3), lo2(pv));
  const float2 h = half_update(d2, hi2(own), t2, hi2(n1), hi2(n2), hi2(n3), hi2(pv));
  return make_float4(l.x, l.y, h.x, h.y);
}

// Moment terms of one level for the two states of a pair, a = phi_j and n = phi_{j+1}:
// <phi_j|phi_j> and Re<phi_{j+1}|phi_j> as packed (re, im) halves, summed at the fold.  For a
// Hermitian H~, <phi_{j+1}|phi_j> = <psi|T_{j+1}(H~) T_j(H~)|psi> is real (the two polynomials
// commute and are Hermitian), so its imaginary part is not accumulated.
// acc2[0] = |a_0|^2, acc2[1] = |a_1|^2, acc2[2] = Re n_0^* a_0, acc2[3] = Re n_1^* a_1 (halves)
__device__ __forceinline__ void moment_terms(float2* acc2, float4 a, float4 n) {
  acc2[0] = __ffma2_rn(lo2(a), lo2(a), acc2[0]);
  acc2[1] = __ffma2_rn(hi2(a), hi2(a), acc2[1]);
  acc2[2] = __ffma2_rn(lo2(n), lo2(a), acc2[2]);
  acc2[3] = __ffma2_rn(hi2(n), hi2(a), acc2[3]);
}

// WIN: window mode for the time blocks -- every level goes to its own buffer (a.win[L-1]) and no
// moment is summed; otherwise levels K-1 and K go to prev_out, cur_out with the moments.
template <int NT_, int K_, int NSLOT_, bool HAS_DIAG, bool OPEN, bool WIN = false>
__global__ void __launch_bounds__(NT_, Cfg<NT_, K_, NSLOT_>::MINB) k_sweep_moments(Args a) {
  using C = Cfg<NT_, K_, NSLOT_>;
  constexpr int NT = C::NT, K = C::K, H = C::H, NSLOT = C::NSLOT, NV = C::NV;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ unsigned ticket;
  const int P = a.P, logP = a.logP, CW = a.CW;
  const int SU = C::slot_units(P), XU = 2 * NT + P;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smraw);
  float4* ring = reinterpret_cast<float4*>(smraw + C::BAR_BYTES);  // [NSLOT][SU]
  float4* xb = ring + NSLOT * SU;                                   // [K-1][2][XU]
  double* red = reinterpret_cast<double*>(xb + 2 * (K - 1) * XU);   // [warps][P][NV]
  float2* dring = reinterpret_cast<float2*>(red + (NT / 32) * P * NV);  // [4][NT] (disorder only)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);

  for (int i = tid; i < NSLOT * SU + 2 * (K - 1) * XU; i += NT) ring[i] = zero;
  for (int i = tid; i < (NT / 32) * P * NV; i += NT) red[i] = 0.0;
  if (tid == 0) {
    for (int s = 0; s < NSLOT; ++s) mbar_init(smem_u32(bars + s), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // the zero pads written through the generic proxy must be ordered before the bulk copies
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();

  const int bx = blockIdx.x % a.nbx, sy = blockIdx.x / a.nbx;
  const int64_t x0 = (int64_t)bx * a.BX;
  const int64_t ys = (int64_t)sy * a.SY;
  const int64_t ye = ys + a.SY < a.Ly ? ys + a.SY : a.Ly;
  const int64_t r0 = ys - H;          // first sweep position = first level-0 row
  const int64_t rlast = ye + H - 1;   // last level-0 row any exact value needs
  const int ny = (int)(ye - ys);
  const int npos = ny + K - 1 + H;    // positions r0 .. ye + K - 2 (level K reaches row ye - 1)
  const int64_t row_units = 2 * a.Lx * P;
  // level-0 rows that hold data, as local indices i = row - r0: [v_lo, v_hi]
  const bool open_y = OPEN && !a.pbc_y;
  const int v_lo = (open_y && r0 < 0) ? (int)(-r0) : 0;
  const int v_hi = (int)(((open_y && rlast > a.Ly - 1) ? a.Ly - 1 : rlast) - r0);

  // this thread's cell and pair.  The band [x0 - H, x0 - H + CW) and the rows r0 .. r_end lie
  // within one period of the lattice on either side (the host requires Lx >= CW, Ly > H), so a
  // single wrap brings any coordinate back into it.
  const int c = tid >> logP, p = tid & (P - 1);
  int64_t x = x0 - H + c;
  bool ghx = false;
  if (x < 0 || x >= a.Lx) {
    if (OPEN && !a.pbc_x) ghx = true;
    else x = x < 0 ? x + a.Lx : x - a.Lx;
  }
  const bool intx = c >= H && c < CW - H && x0 + c - H < a.Lx;
  const int64_t colA = 2 * x * P + p;
  const int uA = 2 * (c << logP) + p;  // unit of A(c, pair p) in a ring row; B is + P
  const int wA = tid, wB = NT + P + tid;
  // Ring rows interleave A and B per cell, so the A units of the cells of a quarter-warp share
  // banks.  Threads with bit 2 of tid set take each pair of level-0 loads in the opposite order,
  // which puts the two halves of a quarter-warp on different banks for any P.
  const bool swp = (tid >> 2) & 1;
  const int o_pvA = 2 * NT + P + uA, o_pvB = o_pvA + P;  // phi_{n-1} A, B of row r (R0)
  const int o_bxm = uA - P, o_axp = uA + 2 * P;          // B(x-1, r), A(x+1, r) (R0)
  const int o_p1 = swp ? o_pvB : o_pvA, o_p2 = swp ? o_pvA : o_pvB;
  const int o_n1 = swp ? o_axp : o_bxm, o_n2 = swp ? o_bxm : o_axp;

  // row index in the lattice of local row i, or -1 where the row holds no data
  auto grow = [&](int i) -> int64_t {
    if (i < v_lo || i > v_hi) return -1;
    const int64_t r = r0 + i;
    if (r >= 0 && r < a.Ly) return r;
    return r < 0 ? r + a.Ly : r - a.Ly;
  };

  // producer (thread 0): the band's pieces inside the lattice are the same for every row (at
  // most two: one wrap when periodic); rows are issued in order, slot after slot; a row without
  // data is filled with zeros from g_zero_rows
  int pc0 = 0, pn0 = 0, pc1 = 0, pn1 = 0;
  int64_t pg0 = 0, pg1 = 0;
  if (!a.pbc_x) {
    const int64_t lo = H - x0 > 0 ? H - x0 : 0;
    const int64_t hi = a.Lx - x0 + H < CW ? a.Lx - x0 + H : CW;
    if (lo < hi) {
      pc0 = (int)lo;
      pg0 = x0 - H + lo;
      pn0 = (int)(hi - lo);
    }
  } else {
    pg0 = x0 - H < 0 ? x0 - H + a.Lx : x0 - H;
    pn0 = (int)(a.Lx - pg0 < CW ? a.Lx - pg0 : CW);
    pc1 = pn0;
    pg1 = 0;
    pn1 = CW - pn0;
  }
  const uint32_t piece_bytes0 = (uint32_t)pn0 * 2u * (uint32_t)P * 16u;
  const uint32_t piece_bytes1 = (uint32_t)pn1 * 2u * (uint32_t)P * 16u;
  const uint32_t zero_bytes = 2u * NT * 16u;
  int next_row = 0;  // local index of the next row to issue
  int next_slot = 0;
  // rows 0 .. npos are read (row r+1 at the last position); none beyond is issued, so no copy is
  // in flight when the CTA finishes its sweep
  auto issue_next = [&]() {
    if (next_row > npos) return;
    const int j = next_row;
    const int slot = next_slot;
    ++next_row;
    next_slot = next_slot + 1 == NSLOT ? 0 : next_slot + 1;
    const uint32_t bar = smem_u32(bars + slot);
    const uint32_t sn = smem_u32(ring + slot * SU + P);
    const uint32_t sp = smem_u32(ring + slot * SU + 2 * NT + 2 * P);
    const int64_t gy = grow(j);
    if (gy < 0) {
      mbar_arrive_tx(bar, 2u * zero_bytes);
      bulk_g2s(sn, g_zero_rows, zero_bytes, bar);
      bulk_g2s(sp, g_zero_rows, zero_bytes, bar);
      return;
    }
    const int64_t src0 = gy * row_units + pg0 * 2 * P;
    const int64_t src1 = gy * row_units + pg1 * 2 * P;
    if (!TBPM_DBG_OK(src0 + (int64_t)pn0 * 2 * P - 1, a.Ly * row_units, TBPM_DBG_SWEEP_ROW) ||
        (pn1 > 0 && !TBPM_DBG_OK(src1 + (int64_t)pn1 * 2 * P - 1, a.Ly * row_units, TBPM_DBG_SWEEP_ROW))) {
      mbar_arrive(bar);  // debug build: the row is not copied (the kernel's results are void)
      return;
    }
    mbar_arrive_tx(bar, 2u * (piece_bytes0 + piece_bytes1));
    bulk_g2s(sn + 32u * pc0 * P, a.cur_in + src0, piece_bytes0, bar);
    bulk_g2s(sp + 32u * pc0 * P, a.prev_in + src0, piece_bytes0, bar);
    if (pn1 > 0) {
      bulk_g2s(sn + 32u * pc1 * P, a.cur_in + src1, piece_bytes1, bar);
      bulk_g2s(sp + 32u * pc1 * P, a.prev_in + src1, piece_bytes1, bar);
    }
  };
  if (tid == 0)
    for (int k = 0; k < NSLOT; ++k) issue_next();

  const float* drow = HAS_DIAG ? a.diag + 2 * x : nullptr;
  auto diag_row = [&](int i) -> float2 {
    if (!HAS_DIAG) return make_float2(a.dc2, a.dc2);
    const int64_t gy = grow(i);
    if (gy < 0 || ghx) return make_float2(0.f, 0.f);
    const float2 d = __ldg(reinterpret_cast<const float2*>(drow + 2 * gy * a.Lx));
    return make_float2(2.f * d.x, 2.f * d.y);
  };

  // registers: level l = 1 .. K-1 at the rows formed in the last three positions (slot =
  // position % 3); level 0 (phi_n) is read from the ring, which keeps row j until position j + 1
  float4 RA[K][3], RB[K][3];
#pragma unroll
  for (int l = 0; l < K; ++l)
#pragma unroll
    for (int s = 0; s < 3; ++s) RA[l][s] = RB[l][s] = zero;
  float2 acc2[NV];  // packed halves of the NV sums (level L: [4(L-1), 4L))
#pragma unroll
  for (int v = 0; v < NV; ++v) acc2[v] = make_float2(0.f, 0.f);
  int folded = 0;
  // every FOLD positions: the FP32 partials of the lanes of each state pair (lane = p + P m) are
  // reduce-scattered across the lanes (each exchange halves the values a lane keeps), so that a
  // lane ends with 16 / (32 / P) fully summed values and adds only those into the warp's FP64
  // slots: the FP64 work is spread over the whole warp instead of P lanes
  static_assert(NV == 16, "the fold splits 16 values");
  auto fold = [&]() {
    const int pp = lane & (P - 1);
    double* slot = red + (warp * P + pp) * NV;
    float v16[16];
#pragma unroll
    for (int v = 0; v < 16; ++v) {
      v16[v] = acc2[v].x + acc2[v].y;
      acc2[v] = make_float2(0.f, 0.f);
    }
    auto half = [&](const float* in, float* out, int n, int off) {
      const bool up = (lane & off) != 0;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (k < n / 2) {
          const float keep = up ? in[n / 2 + k] : in[k];
          const float send = up ? in[k] : in[n / 2 + k];
          out[k] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
      }
    };
    float v8[8];
    half(v16, v8, 16, 16);
    const int b16 = (lane & 16) ? 8 : 0;
    if (P == 16) {
#pragma unroll
      for (int k = 0; k < 8; ++k) slot[b16 + k] += (double)v8[k];
      return;
    }
    float v4[4];
    half(v8, v4, 8, 8);
    const int b8 = b16 + ((lane & 8) ? 4 : 0);
    if (P == 8) {
#pragma unroll
      for (int k = 0; k < 4; ++k) slot[b8 + k] += (double)v4[k];
      return;
    }
    float v2[2];
    half(v4, v2, 4, 4);
    const int b4 = b8 + ((lane & 4) ? 2 : 0);
    if (P == 4) {
#pragma unroll
      for (int k = 0; k < 2; ++k) slot[b4 + k] += (double)v2[k];
      return;
    }
    float v1[1];
    half(v2, v1, 2, 2);
    const int b2 = b4 + ((lane & 2) ? 1 : 0);
    // P = 2: every lane holds one sum; P = 1: lanes 2k and 2k+1 hold halves of the same one
    if (P == 1) v1[0] += __shfl_xor_sync(0xffffffffu, v1[0], 1);
    if (P == 2 || (lane & 1) == 0) slot[b2] += (double)v1[0];
  };
  // outputs of levels K-1 and K at the rows they form at the current position
  float4* out_km1 = a.prev_out + (r0 - (K - 2)) * row_units + colA;
  float4* out_k = a.cur_out + (r0 - (K - 1)) * row_units + colA;
  int64_t off_r = r0 * row_units + colA;  // window mode: offset of row r in every level's buffer
  // ring slots of level-0 rows r and r+1 (a slot's phi_{n-1} row follows at + 2 NT + P)
  int slot_m1 = 0, slot_0 = 0, slot_p1 = 1 % NSLOT;  // row r0 - 1 stands in as row r0
  uint32_t wait_par = NSLOT == 1 ? 1u : 0u;  // phase parity of row r+1's slot

  // disordered lattices: 2 D of row r in flight, stored into the ring at position r
  float2 dq0 = diag_row(0);
  bool timed_out = !mbar_wait(smem_u32(bars + 0), 0);  // this thread's waits; OR-reduced per position
  // level-0 values carried from position to position: A(r) (loaded as A(x, r+1) one position
  // earlier), A(r-1), B(r-1) (this thread's own cell); row r0 - 1 stands in as row r0
  float4 c0A = ring[P + uA];
  float4 cmA = c0A, cmB = ring[P + uA + P];
  const float th = a.th2;
  bool aborted = false;
  int i_done = -1;  // last position completed

  for (int ib = 0; ib < npos && !aborted; ib += 3) {
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int i = ib + u;
      if (i >= npos || aborted) break;
      const int s0 = u, s1 = (u + 2) % 3, s2 = (u + 1) % 3;  // ages 0, 1, 2
      if (!mbar_wait(smem_u32(bars + slot_p1), wait_par)) timed_out = true;  // level-0 row r+1
      const float4* R0 = ring + slot_0 * SU + P;
      const float4* Rp = ring + slot_p1 * SU + P;
      const float4* Rm_ = ring + slot_m1 * SU + P;  // row r-1 (disordered lattices)
      // x-neighbours of levels 1 .. K-1 written at the previous position, loaded before this
      // position writes the exchange row of the level before (the compiler cannot tell the two
      // parities apart): level 1's right away, the others once level 1 has been stored
      float4 xbm[K], xap[K];
      const float4* Xprev = xb + ((i - 1) & 1) * XU;  // level l at + 2 (l - 1) XU
      xbm[1] = Xprev[wB - P];
      xap[1] = Xprev[wA + P];
      const float4 prevA = cmA, prevB = cmB;  // level-0 row r-1 of this cell
      if (HAS_DIAG) {
        dring[(i & 3) * NT + tid] = dq0;
        dq0 = diag_row(i + 1);
      }
#pragma unroll
      for (int L = 1; L <= K; ++L) {
        const int iq = i - (L - 1);  // local row of this level
        float4 ownA, ownB, bxm, axp, bym, ayp, pvA, pvB;
        if (L == 1) {
          // three pairs of loads, each issued in the thread's bank order
          const float4 q1 = swp ? Rp[uA] : R0[uA + P], q2 = swp ? R0[uA + P] : Rp[uA];
          const float4 n1 = R0[o_n1], n2 = R0[o_n2];
          const float4 p1 = R0[o_p1], p2 = R0[o_p2];
          // disordered lattices: level-0 values of rows r and r-1 from the ring (the registers
          // that would carry them go to the diagonal's prefetch)
          ownA = HAS_DIAG ? R0[uA] : c0A;
          ownB = swp ? q2 : q1;
          ayp = swp ? q1 : q2;
          bxm = swp ? n2 : n1;
          axp = swp ? n1 : n2;
          pvA = swp ? p2 : p1;
          pvB = swp ? p1 : p2;
          bym = HAS_DIAG ? Rm_[uA + P] : prevB;
          cmA = ownA;  // carried to the next position: row r becomes row r-1, A(r+1) becomes A(r)
          cmB = ownB;
          c0A = ayp;
        } else {
          ownA = RA[L - 1][s1];
          ownB = RB[L - 1][s1];
          bxm = xbm[L - 1];
          axp = xap[L - 1];
          bym = RB[L - 1][s2];
          ayp = RA[L - 1][s0];
          if (L == 2) {
            pvA = HAS_DIAG ? Rm_[uA] : prevA;
            pvB = HAS_DIAG ? Rm_[uA + P] : prevB;
          } else {
            pvA = RA[L - 2][s2];
            pvB = RB[L - 2][s2];
          }
        }
        // disordered lattices: 2 D of this level's row from the thread's own ring
        const float2 dl = HAS_DIAG ? dring[(iq & 3) * NT + tid] : make_float2(a.dc2, a.dc2);
        const float dA = dl.x, dB = dl.y;
        float4 nA = level_update(dA, ownA, th, ownB, bxm, bym, pvA);
        float4 nB = level_update(dB, ownB, th, ownA, axp, ayp, pvB);
        if (OPEN && (ghx || iq < v_lo || iq > v_hi)) {
          nA = zero;
          nB = zero;
        }
        if (L < K) {
          RA[L][s0] = nA;
          RB[L][s0] = nB;
          float4* Xout = xb + ((L - 1) * 2 + (i & 1)) * XU;
          Xout[wA] = nA;
          Xout[wB] = nB;
        }
        if (L == 1) {
#pragma unroll
          for (int l = 2; l < K; ++l) {
            xbm[l] = Xprev[2 * (l - 1) * XU + wB - P];
            xap[l] = Xprev[2 * (l - 1) * XU + wA + P];
          }
        }
        if (intx && (unsigned)(iq - H) < (unsigned)ny &&
            TBPM_DBG_OK(off_r - (int64_t)(L - 1) * row_units, a.Ly * row_units, TBPM_DBG_SWEEP_STORE)) {
          if (WIN) {
            float4* dst = a.win[L - 1] + (off_r - (int64_t)(L - 1) * row_units);
            __stcs(dst, nA);
            __stcs(dst + P, nB);
          } else {
            if (L == K - 1) {
              __stcs(out_km1, nA);
              __stcs(out_km1 + P, nB);
            } else if (L == K) {
              __stcs(out_k, nA);
              __stcs(out_k + P, nB);
            }
            moment_terms(acc2 + (L - 1) * 4, ownA, nA);
            moment_terms(acc2 + (L - 1) * 4, ownB, nB);
          }
        }
      }
      off_r += row_units;
      if (!WIN) {
        out_km1 += row_units;
        out_k += row_units;
        if (++folded == C::FOLD) {
          folded = 0;
          fold();
        }
      }
      // one barrier per position; it also tells every thread whether any wait expired
      if (__syncthreads_or(timed_out ? 1 : 0)) {
        aborted = true;
        break;
      }
      i_done = i;
      // row r-1 has been read for the last time: refill its slot with row r - 1 + NSLOT
      if (tid == 0 && i >= 1) issue_next();
      slot_m1 = slot_0;
      slot_0 = slot_p1;
      slot_p1 = slot_p1 + 1 == NSLOT ? 0 : slot_p1 + 1;
      if (slot_p1 == 0) wait_par ^= 1u;
    }
  }
  if (aborted && tid == 0) {
    // copies in flight into this CTA's shared memory must land before it exits: rows
    // i_done + 2 .. next_row - 1 were issued and never waited for (bounded waits)
    bool err_wait = false;
    for (int j = i_done + 2 > 0 ? i_done + 2 : 0; j < next_row; ++j)
      if (!mbar_wait(smem_u32(bars + j % NSLOT), (uint32_t)((j / NSLOT) & 1))) err_wait = true;
    atomicExch(a.status, err_wait ? 2 : 1);
  }
  if (WIN) return;
  fold();
  __syncthreads();
  for (int qv = tid; qv < P * NV; qv += NT) {  // warps in order
    const int pp = qv / NV, v = qv - pp * NV;
    double t = 0.0;
    for (int w = 0; w < NT / 32; ++w) t += red[(w * P + pp) * NV + v];
    a.partials[(size_t)blockIdx.x * P * NV + qv] = t;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) ticket = atomicAdd(a.counter, 1u);
  __syncthreads();
  if (ticket != gridDim.x - 1) return;
  __threadfence();
  const int nval = K * a.S * 2;
  for (int v = warp; v < nval; v += NT / 32) {
    const int k = v / (a.S * 2), rem = v - k * a.S * 2, s = rem / 2, comp = rem - s * 2;
    const int pr = s >> 1, sub = s & 1;
    const int idx = k * 4 + comp * 2 + sub;
    double sum = 0.0;
    for (int t = lane; t < (int)gridDim.x; t += 32) sum += __ldcg(a.partials + ((size_t)t * P + pr) * NV + idx);
    for (int off = 16; off >= 1; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
    if (lane == 0) {
      const int j = a.step0 + k;
      double* ms = a.mu + (size_t)s * a.M * 2;
      if (comp == 0) {  // m_{2j} = 2 <phi_j|phi_j> - m_0 (real)
        ms[4 * j] = 2.0 * sum - ms[0];
        ms[4 * j + 1] = -ms[1];
      } else {          // m_{2j+1} = 2 <phi_{j+1}|phi_j> - m_1, the inner product real
        ms[4 * j + 2] = 2.0 * sum - ms[2];
        ms[4 * j + 3] = -ms[3];
      }
    }
  }
  if (tid == 0) *a.counter = 0u;
}

// Expiry check of the bounded wait above: one warp waits on an mbarrier of its own that expects
// one arrival.  With `arrive`, thread 0 arrives first and the phase completes; without it nothing
// ever arrives, no copy is in flight, and every thread's wait gives up after budget_ns.  An
// expired wait is reported as the sweep reports one: code 1 in the caller's status word.
__global__ void __launch_bounds__(32) k_wait_probe(int* status, uint64_t budget_ns, int arrive) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t b = smem_u32(&bar);
  if (threadIdx.x == 0) {
    mbar_init(b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (arrive && threadIdx.x == 0) mbar_arrive(b);
  const bool done = mbar_wait_ns(b, 0, budget_ns);
  if (__syncthreads_or(done ? 0 : 1) && threadIdx.x == 0) atomicExch(status, 1);
}

}  // namespace sweep

template <int NT, int K, int NSLOT, bool D, bool O, bool W = false>
static cudaError_t set_sweep_smem() {
  return cudaFuncSetAttribute(sweep::k_sweep_moments<NT, K, NSLOT, D, O, W>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sweep::Cfg<NT, K, NSLOT>::smem(16, true));
}

// win != null: window mode, phi_{n+1..n+4} into win[0..3] (no moments)
template <int NT, int K, int NSLOT>
static int launch_sweep(tbpm_ctx* ctx, const tbpm_lattice* lat, const RecurrenceArgs& ra, const void* prev_in,
                        const void* cur_in, void* prev_out, void* cur_out, int step0, void* const* win = nullptr) {
  using namespace sweep;
  using Cf = Cfg<NT, K, NSLOT>;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    cudaError_t e[8] = {set_sweep_smem<NT, K, NSLOT, false, false>(), set_sweep_smem<NT, K, NSLOT, false, true>(),
                        set_sweep_smem<NT, K, NSLOT, true, false>(), set_sweep_smem<NT, K, NSLOT, true, true>(),
                        set_sweep_smem<NT, K, NSLOT, false, false, true>(),
                        set_sweep_smem<NT, K, NSLOT, false, true, true>(),
                        set_sweep_smem<NT, K, NSLOT, true, false, true>(),
                        set_sweep_smem<NT, K, NSLOT, true, true, true>()};
    for (cudaError_t x : e)
      if (x != cudaSuccess) attr = x;
  });
  TBPM_CK(attr);
  if (ctx->pinned_cap < 256) {
    set_error("context has no pinned status word");
    return TBPM_ECUDA;
  }
  Args a;
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
  a.CW = NT / a.P;
  a.BX = a.CW - 2 * Cf::H;
  if (a.BX < 1) {
    set_error("fused sweep: band too narrow for %d states", a.S);
    return TBPM_EUNSUPPORTED;
  }
  a.nbx = (int)((a.Lx + a.BX - 1) / a.BX);
  static int per_sm = 0;
  if (per_sm == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_moments<NT, K, NSLOT, false, false>, NT,
                                                      Cf::smem(4, false)) != cudaSuccess || per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
  }
  // segments per band: the count whose CTAs fill the resident slots best over whole waves, weighed
  // by the sweep positions each segment adds (K/2 halo rows at each end, K - 1 to drain)
  const int64_t slots = (int64_t)ctx->num_sms * per_sm;
  const int64_t max_nsy = std::max<int64_t>(1, std::min<int64_t>(a.Ly / 4, 8 * slots / a.nbx + 1));
  int64_t nsy = 1;
  double best = -1.0;
  for (int64_t k = 1; k <= max_nsy; ++k) {
    const int64_t sy = (a.Ly + k - 1) / k;
    const int64_t ctas = a.nbx * ((a.Ly + sy - 1) / sy);
    const int64_t waves = (ctas + slots - 1) / slots;
    const double eff = (double)ctas / (double)(waves * slots) * (double)sy / (double)(sy + 2 * K);
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
  a.status = reinterpret_cast<int*>(ctx->pinned + kSweepStatusSlot);
  const int64_t grid = (int64_t)a.nbx * a.nsy;
  TBPM_TRY(ensure(ctx, ctx->ws_fused_partials, sizeof(double) * Cf::NV * (size_t)a.P * (size_t)grid));
  a.partials = (double*)ctx->ws_fused_partials.p;
  a.counter = ra.counter;
  const bool open = !(a.pbc_x && a.pbc_y);
  const dim3 gr((unsigned)grid), bl(NT);
  const size_t sm = Cf::smem(a.P, a.diag != nullptr);
  if (win) {
    for (int l = 0; l < 4; ++l) a.win[l] = (float4*)win[l];
    if (a.diag) {
      if (open) k_sweep_moments<NT, K, NSLOT, true, true, true><<<gr, bl, sm, ctx->stream>>>(a);
      else k_sweep_moments<NT, K, NSLOT, true, false, true><<<gr, bl, sm, ctx->stream>>>(a);
    } else {
      if (open) k_sweep_moments<NT, K, NSLOT, false, true, true><<<gr, bl, sm, ctx->stream>>>(a);
      else k_sweep_moments<NT, K, NSLOT, false, false, true><<<gr, bl, sm, ctx->stream>>>(a);
    }
  } else if (a.diag) {
    if (open) k_sweep_moments<NT, K, NSLOT, true, true><<<gr, bl, sm, ctx->stream>>>(a);
    else k_sweep_moments<NT, K, NSLOT, true, false><<<gr, bl, sm, ctx->stream>>>(a);
  } else {
    if (open) k_sweep_moments<NT, K, NSLOT, false, true><<<gr, bl, sm, ctx->stream>>>(a);
    else k_sweep_moments<NT, K, NSLOT, false, false><<<gr, bl, sm, ctx->stream>>>(a);
  }
  TBPM_CK_LAUNCH(ctx);
  return TBPM_OK;
}

// Window pass of the time blocks: phi_{n+1} .. phi_{n+4} from (prev_in = phi_{n-1}, cur_in = phi_n)
// into win[0..3] by the 128-thread register sweep; false when the lattice does not take it.
bool sweep_window_applicable(const tbpm_lattice* lat, int precision, int Spad) {
  return fused_applicable(lat, precision, Spad) && lat->geom.Lx >= 128 / (Spad / 2);
}

int launch_sweep_window(tbpm_ctx* ctx, const tbpm_lattice* lat, const RecurrenceArgs& ra, const void* prev_in,
                        const void* cur_in, void* const win[4]) {
  return launch_sweep<128, 4, 5>(ctx, lat, ra, prev_in, cur_in, nullptr, nullptr, 0, win);
}

// One register-resident sweep pass: steps step0 .. step0+K-1 from (prev_in, cur_in) into
// (prev_out, cur_out).  Variant 8: 128 threads; 9: 192 threads; 10: 256 threads (K = 4).
int launch_sweep_pass(tbpm_ctx* ctx, const tbpm_lattice* lat, const RecurrenceArgs& ra, const void* prev_in,
                      const void* cur_in, void* prev_out, void* cur_out, int step0, int variant) {
  if (variant == 9) return launch_sweep<192, 4, 4>(ctx, lat, ra, prev_in, cur_in, prev_out, cur_out, step0);
  if (variant == 10) return launch_sweep<256, 4, 4>(ctx, lat, ra, prev_in, cur_in, prev_out, cur_out, step0);
  return launch_sweep<128, 4, 5>(ctx, lat, ra, prev_in, cur_in, prev_out, cur_out, step0);
}

int sweep_status(tbpm_ctx* ctx) {
  int* st = reinterpret_cast<int*>(ctx->pinned + kSweepStatusSlot);
  const int v = *st;
  if (v != 0) {
    *st = 0;
    set_error("fused sweep: a bounded wait for a row copy expired (code %d)", v);
    return TBPM_ETIMEOUT;
  }
  return TBPM_OK;
}

}  // namespace tbpm

TBPM_DEBUG_UNIT(sweep)

using namespace tbpm;

// One-warp run of the register sweep's bounded mbarrier wait, reported through the sweep's status
// word and sweep_status(): TBPM_ETIMEOUT when the wait expired.
extern "C" int tbpm_wait_probe(tbpm_ctx* ctx, int arrive, double budget_s) {
  clear_error();
  if (!ctx) {
    set_error("tbpm_wait_probe: NULL context");
    return TBPM_EINVAL;
  }
  if (!(budget_s > 0.0 && budget_s <= 2.0)) {
    set_error("tbpm_wait_probe: budget %g s outside (0, 2]", budget_s);
    return TBPM_EINVAL;
  }
  if (ctx->pinned_cap < 256) {
    set_error("context has no pinned status word");
    return TBPM_ECUDA;
  }
  TBPM_CK(cudaSetDevice(ctx->device));
  int* status = reinterpret_cast<int*>(ctx->pinned + kSweepStatusSlot);
  const uint64_t budget_ns = (uint64_t)(budget_s * 1e9);
  sweep::k_wait_probe<<<1, 32, 0, ctx->stream>>>(status, budget_ns, arrive ? 1 : 0);
  TBPM_CK_LAUNCH(ctx);
  TBPM_CK(cudaStreamSynchronize(ctx->stream));
  return sweep_status(ctx);
}
