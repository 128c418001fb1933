// Internal declarations shared by the library's translation units.
//
// Device-side building blocks:
//   * Philox4x32-10 (Salmon et al., SC'11): the counter-based generator behind the
//     disorder, vacancy and random-phase draws.
//   * lattice geometry: full site index -> neighbour full index for the square,
//     honeycomb and simple-cubic stencils in their fixed neighbour order.
//   * the grid-wide deterministic reduction used by every fused inner product:
//     per-thread compensated FP32 sums -> FP64 warp/block trees -> per-block partials
//     -> the last block to finish sums the partials in block order.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/tbpm.h"

// ------------------------------------------------------------------ debug builds (TBPM_DEBUG)
// A debug build (libtbpm_debug.so) checks the global-memory indices of the hot kernels: an index
// outside its buffer is not accessed, and the first one is recorded in a device status word of
// the translation unit ((kernel id << 48) | (index & 0xFFFFFFFFFFFF)); there is no trap, so the
// context stays usable.  tbpm_debug_status() collects and clears the words of every unit.  In
// the regular build the checks compile to nothing.
enum {
  TBPM_DBG_STENCIL = 1,     // k_moment_stencil: own and neighbour units
  TBPM_DBG_ELL = 2,         // ELL neighbour index against the site count
  TBPM_DBG_SWEEP_STORE = 3, // k_sweep_moments: output units
  TBPM_DBG_SWEEP_ROW = 4,   // k_sweep_moments: source range of a row copy
  TBPM_DBG_SERVE = 5        // k_serve_step: neighbour units
};
#ifdef TBPM_DEBUG
static __device__ unsigned long long g_tbpm_dbg;
__device__ __forceinline__ bool tbpm_dbg_ok(int64_t idx, int64_t n, int kid) {
  if ((uint64_t)idx < (uint64_t)n) return true;
  atomicCAS(&g_tbpm_dbg, 0ull, ((unsigned long long)kid << 48) | ((unsigned long long)idx & 0xFFFFFFFFFFFFull));
  return false;
}
#define TBPM_DBG_OK(idx, n, kid) tbpm_dbg_ok((int64_t)(idx), (int64_t)(n), (kid))
// host accessor of a unit's word (reads and clears it on the current device)
#define TBPM_DEBUG_UNIT(name)                                                      \
  namespace tbpm {                                                                 \
  unsigned long long debug_take_##name() {                                         \
    unsigned long long v = 0, z = 0;                                               \
    if (cudaMemcpyFromSymbol(&v, g_tbpm_dbg, sizeof(v)) != cudaSuccess) v = ~0ull; \
    cudaMemcpyToSymbol(g_tbpm_dbg, &z, sizeof(z));                                 \
    return v;                                                                      \
  }                                                                                \
  }
#else
#define TBPM_DBG_OK(idx, n, kid) true
#define TBPM_DEBUG_UNIT(name)
#endif

namespace tbpm {

#ifdef TBPM_DEBUG
unsigned long long debug_take_cheb();
unsigned long long debug_take_sweep();
unsigned long long debug_take_serve();
#endif

// ------------------------------------------------------------------ error reporting
void set_error(const char* fmt, ...);
void clear_error();

#define TBPM_CK(call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      ::tbpm::set_error("%s:%d %s: %s", __FILE_NAME__, __LINE__, #call, cudaGetErrorString(e_)); \
      return TBPM_ECUDA;                                                               \
    }                                                                                  \
  } while (0)

#define TBPM_CK_LAUNCH(ctx)                                                            \
  do {                                                                                 \
    (ctx)->launches++;                                                                 \
    cudaError_t e_ = cudaGetLastError();                                               \
    if (e_ != cudaSuccess) {                                                           \
      ::tbpm::set_error("%s:%d kernel launch: %s", __FILE_NAME__, __LINE__, cudaGetErrorString(e_)); \
      return TBPM_ECUDA;                                                               \
    }                                                                                  \
  } while (0)

#define TBPM_TRY(expr)            \
  do {                            \
    int r_ = (expr);              \
    if (r_ != TBPM_OK) return r_; \
  } while (0)

// ------------------------------------------------------------------ Philox4x32-10
__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

// 10 rounds of the Philox S-box: (c0,c1,c2,c3) -> (hi(M1 c2)^c1^k0, lo(M1 c2), hi(M0 c0)^c3^k1, lo(M0 c0)),
// key advanced by the Weyl constants between rounds.
__host__ __device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = mulhi32(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = mulhi32(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

enum { STREAM_DISORDER = 0, STREAM_VACANCY = 1, STREAM_PHASE = 2 };

// First output word at counter (index, stream, sub) under the 64-bit seed.
__host__ __device__ __forceinline__ uint32_t draw_u32(uint64_t seed, uint64_t index, uint32_t stream,
                                                      uint32_t sub) {
  return philox10(make_uint4((uint32_t)index, (uint32_t)(index >> 32), stream, sub), (uint32_t)seed,
                  (uint32_t)(seed >> 32))
      .x;
}

// ------------------------------------------------------------------ lattice geometry
struct Geom {
  int kind;          // TBPM_SQUARE / TBPM_HONEYCOMB / TBPM_CUBIC
  int64_t Lx, Ly, Lz;
  int pbc_x, pbc_y, pbc_z;
  int z;             // coordination
  int64_t n_full;
  int64_t row_sites; // sites on one x-line: Lx, or 2*Lx for the honeycomb
  int64_t n_rows;    // Ly * Lz
};

__host__ __device__ __forceinline__ int64_t wrap_coord(int64_t v, int64_t n, int periodic, bool* ok) {
  if (v < 0) {
    if (!periodic) { *ok = false; return 0; }
    return v + n;
  }
  if (v >= n) {
    if (!periodic) { *ok = false; return 0; }
    return v - n;
  }
  return v;
}

// Neighbour d (fixed order) of full site i, or -1 when an open boundary drops it.
__host__ __device__ __forceinline__ int64_t neighbour_full(const Geom& g, int64_t i, int d) {
  bool ok = true;
  if (g.kind == TBPM_SQUARE) {
    const int64_t x = i % g.Lx, y = i / g.Lx;
    const int dx = (d == 0) ? 1 : (d == 1) ? -1 : 0;
    const int dy = (d == 2) ? 1 : (d == 3) ? -1 : 0;
    const int64_t xx = wrap_coord(x + dx, g.Lx, g.pbc_x, &ok);
    const int64_t yy = wrap_coord(y + dy, g.Ly, g.pbc_y, &ok);
    return ok ? yy * g.Lx + xx : -1;
  } else if (g.kind == TBPM_HONEYCOMB) {
    const int64_t s = i & 1, c = i >> 1;
    const int64_t x = c % g.Lx, y = c / g.Lx;
    // A: B(x,y), B(x-1,y), B(x,y-1);  B: A(x,y), A(x+1,y), A(x,y+1)
    const int sg = s == 0 ? -1 : 1;
    const int dx = (d == 1) ? sg : 0;
    const int dy = (d == 2) ? sg : 0;
    const int64_t xx = wrap_coord(x + dx, g.Lx, g.pbc_x, &ok);
    const int64_t yy = wrap_coord(y + dy, g.Ly, g.pbc_y, &ok);
    return ok ? 2 * (yy * g.Lx + xx) + (1 - s) : -1;
  } else {
    const int64_t x = i % g.Lx, y = (i / g.Lx) % g.Ly, zc = i / (g.Lx * g.Ly);
    const int dx = (d == 0) ? 1 : (d == 1) ? -1 : 0;
    const int dy = (d == 2) ? 1 : (d == 3) ? -1 : 0;
    const int dz = (d == 4) ? 1 : (d == 5) ? -1 : 0;
    const int64_t xx = wrap_coord(x + dx, g.Lx, g.pbc_x, &ok);
    const int64_t yy = wrap_coord(y + dy, g.Ly, g.pbc_y, &ok);
    const int64_t zz = wrap_coord(zc + dz, g.Lz, g.pbc_z, &ok);
    return ok ? (zz * g.Ly + yy) * g.Lx + xx : -1;
  }
}

// ------------------------------------------------------------------ context & lattice
struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

}  // namespace tbpm

struct tbpm_ctx {
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  int64_t launches = 0;
  // cached workspaces (grow-only, stream-ordered allocations)
  tbpm::DevBuf ws_phi[2], ws_psi, ws_acc, ws_partials, ws_counter, ws_mu, ws_table, ws_aux, ws_out,
      ws_energies, ws_recon, ws_phi2[2], ws_fused_partials, ws_qe, ws_qe_coef, ws_xdot, ws_jpsi, ws_ec, ws_fermi, ws_blk, ws_blk_coef;
  // time blocks buffer up to 32 Chebyshev vectors and flush them into the accumulators at once
  bool buffer_blocks = true;
  int fusion = 8;  // temporal-fusion mode of the moment pass (8 = four-step register sweep; -1 = autotuned)
  // autotuned fusion modes: key (kind, Lx, Ly, Lz, pbc bits, path, Spad, precision, disorder) -> mode
  std::vector<std::pair<std::vector<int64_t>, int>> fusion_choice;
  std::vector<std::pair<int, double>> fusion_timings;  // last autotune: (mode, ms per step)
  // CUDA graphs of moment-pass sequences: a sequence seen twice with the same key (buffers,
  // lattice, sizes, mode) is captured once and replayed afterwards
  struct Graph {
    std::vector<uint64_t> key;
    cudaGraphExec_t exec;
    int64_t kernels;
  };
  bool use_graphs = true;
  std::vector<Graph> graphs;
  std::vector<std::vector<uint64_t>> graph_seen;
  int max_pass_states = 0;  // cap on states per pass of the OC, DP and CD drivers (0 = by memory)
  double* pinned = nullptr;
  size_t pinned_cap = 0;
  // phase timing with CUDA events on the context stream (tbpm_profile)
  // bounded launch queue (0 = unbounded): an eager moment sequence waits, every 64 launches, for
  // the launches enqueued two windows earlier, so that a long sequence never fills the driver's
  // launch queue (serving lanes run beside other streams)
  int max_queue = 0;
  int64_t queue_count = 0;
  cudaEvent_t queue_ev[2] = {nullptr, nullptr};
  bool queue_live[2] = {false, false};
  bool profiling = false;
  struct Phase {
    cudaEvent_t a, b;
    int kind;        // 0 = recurrence, 1 = reconstruction
    int64_t launches;
  };
  std::vector<Phase> phases;
  std::vector<cudaEvent_t> event_pool;
  // NVTX phase ranges open on this context, innermost last (closed by phase_end, or by the
  // public call's NvtxCall when an error path skipped phase_end)
  std::vector<nvtxRangeId_t> nvtx_open;
};

// One piece of a column run of long-range taps for the matrix-free tap kernel: the taps
// (dx, dy0 + k, ds), k < n (1 <= n <= 8), of one destination sublattice, with weights t_k/t
// (0 where the run has a hole or the piece is padded).
struct TapChunk {
  int dx, dy0, ds, n;
  float w[8];
};

struct tbpm_lattice {
  tbpm_ctx* ctx = nullptr;
  tbpm_lattice_desc desc{};
  tbpm::Geom geom{};
  int path = TBPM_PATH_STENCIL;
  int64_t n_sites = 0;
  int64_t n_bonds = 0;
  double E_min = 0, E_max = 0, H0 = 0, half = 1;
  bool has_v = false;
  // rescaled on-site terms D_i = (V_i - H0)/|H| per active site (FP32 and FP64 copies)
  float* d32 = nullptr;
  double* d64 = nullptr;
  double* v64 = nullptr;       // raw V_i (FP64) per active site, for export
  // CSR/ELL path: compact neighbour lists [n_sites][z] (-1 = none)
  int32_t* ell = nullptr;
  // long-range hopping: per-slot weights t_k / t (slot k of every ELL list), FP32 and FP64;
  // null on nearest-neighbour lattices (every bond t)
  float* wrel32 = nullptr;
  double* wrel64 = nullptr;
  std::vector<int> tap_off;      // [z][4] (dx, dy, dz, ds) of each slot (long-range only)
  std::vector<double> tap_t;     // [z] t(r) of each slot (long-range only)
  double* jw = nullptr;          // [3 directions][2 sublattices][z] t_k (r_j - r_i)_a of each slot
  // matrix-free tap kernel (clean long-range square / honeycomb lattices): column-run pieces
  // of destination sublattice 0 then 1 on the device, their counts and the tile halo
  TapChunk* chunks = nullptr;
  int n_chunks[2] = {0, 0};
  int halo_x = 0, halo_y = 0;
  bool tap_exact = false;        // run pieces of every length 1..8 (else 8, 4, 2, 1)
  int64_t* compact = nullptr;  // [n_full] compact index or -1 (CSR path only)
  int64_t* full_of = nullptr;  // [n_sites] full index of each compact site (CSR path only)
};

namespace tbpm {

// grow-only device workspace on the context stream
int ensure(tbpm_ctx* ctx, DevBuf& b, size_t bytes);

// phase timing: begin returns a token (-1 when profiling is off); end closes it.  Both also open
// and close an NVTX range named after the phase, whether or not profiling is on.
int phase_begin(tbpm_ctx* ctx, int kind);
void phase_end(tbpm_ctx* ctx, int token);

// NVTX range over the scope of a public call, named after it, on the calling thread; phase
// ranges opened inside the call and left open by an error return are closed with it.  NVTX
// calls do nothing unless a profiler (ncu, nsys) has attached its handler.
struct NvtxCall {
  tbpm_ctx* ctx;
  size_t depth;
  NvtxCall(tbpm_ctx* c, const char* name) : ctx(c), depth(c ? c->nvtx_open.size() : 0) { nvtxRangePushA(name); }
  ~NvtxCall() {
    while (ctx && ctx->nvtx_open.size() > depth) {
      nvtxRangeEnd(ctx->nvtx_open.back());
      ctx->nvtx_open.pop_back();
    }
    nvtxRangePop();
  }
  NvtxCall(const NvtxCall&) = delete;
  NvtxCall& operator=(const NvtxCall&) = delete;
};
#define TBPM_NVTX_CALL(ctx) ::tbpm::NvtxCall tbpm_nvtx_call_((ctx), __func__)

// ------------------------------------------------------------------ launch plumbing
struct RecurrenceArgs {
  // states
  const void* cur;     // phi_n      [n_sites][S]
  void* prev_out;      // phi_{n-1} in, phi_{n+1} out
  void* next;          // accumulation passes: phi_{n+1} goes here instead (null: into prev_out)
  // lattice
  Geom geom;
  int path;
  const int32_t* ell;  // CSR/ELL neighbour lists
  const void* wrel;    // per-slot weights t_k/t (float* or double*), or null (every bond t)
  // matrix-free tap kernel (complex64, >= 2 states): chunk table, counts, halo, partial sums
  const TapChunk* taps;
  int taps_n0, taps_n1, taps_rx, taps_ry, taps_exact;
  double* tap_partials;
  const void* diag;    // per-site D_i (float* or double*), or null when the lattice is clean
  double diag_const;   // D when diag == null
  double thop;         // t / |H|
  // the same coefficients pre-rounded for the FP32 kernels: first term (x1) and regular
  // terms (x2); kept in the argument block so no kernel recomputes them in FP64
  float th1f, th2f, dc1f, dc2f;
  int64_t n_sites;
  // states-per-thread layout: P = S / spt thread units per site
  int S, P, logP;
  int64_t n_tiles;     // work tiles of 256 thread units
  // reduction
  double* partials;
  unsigned* counter;
  int nblocks;
  // moments output (device [S][M][2]) and step index
  double* mu;
  int M;
  int step;
};

struct AccumArgs {
  RecurrenceArgs r;     // recurrence part (cur, prev_out, lattice, reduction buffers)
  void* acc;            // accumulators [b][n_sites][S]
  int64_t acc_stride;   // elements (complex) between accumulators
  const double* coef;   // [n_terms][b] complex (re, im) incl. the exp(-i H0 t) phase
  int b;
  int j_lo;             // first accumulator still active at this term
  int j_done;           // accumulator whose last term this is, or -1
  int first_term;       // 1: write acc = c phi (n == 0) instead of acc += c phi
  const void* psi;      // initial states for <psi|acc_j>
  double* C;            // device [S][n_steps+1][2]
  int C_len;            // n_steps + 1
  int j_global;         // time index of accumulator j_done
};

// fills th1f/th2f/dc1f/dc2f from thop and diag_const
inline void set_float_coefficients(RecurrenceArgs* a) {
  a->th1f = (float)a->thop;
  a->th2f = (float)(2.0 * a->thop);
  a->dc1f = (float)a->diag_const;
  a->dc2f = (float)(2.0 * a->diag_const);
}

int launch_moment_step(tbpm_ctx* ctx, const RecurrenceArgs& a, int precision, bool first);
// matrix-free tap kernel (csrc/taps.cu): chunk table of a clean long-range lattice, the moment
// pass over it, and the size of its per-CTA partial sums
int build_tap_chunks(tbpm_ctx* ctx, tbpm_lattice* lat);
int ensure_ell(tbpm_ctx* ctx, tbpm_lattice* lat);  // ELL lists of a long-range lattice, on first need
int launch_taps_moment(tbpm_ctx* ctx, const RecurrenceArgs& a, bool first);
int launch_taps_step(tbpm_ctx* ctx, const RecurrenceArgs& a, bool first);  // recurrence only
size_t taps_partials_bytes(const RecurrenceArgs& a);
int launch_accum_step(tbpm_ctx* ctx, const AccumArgs& a, int precision, int mode);
// acc_j += sum_{t<T} c_t(j) phi_t over T consecutive buffered state blocks phi and nb
// consecutive accumulators; coef [T][nb] complex (csrc/cheb.cu)
// tile: accumulators per CTA tile (1, 4 or 16); 0 = chosen from nb
int launch_block_flush(tbpm_ctx* ctx, const RecurrenceArgs& a, int precision, const void* phi, int T, void* acc,
                       int nb, const double* coef, int tile = 0);
int launch_dot(tbpm_ctx* ctx, const RecurrenceArgs& a, int precision, const void* x, const void* y,
               double* out /* device [S][2] at stride out_stride */, int out_stride);
int recurrence_blocks(tbpm_ctx* ctx, int precision, int S);
int launch_qe_axpy(tbpm_ctx* ctx, const RecurrenceArgs& a, int precision, const void* x, void* qe,
                   const double* phase, int width, int j, double sgn, double scale, int nE);
int qe_flush_max_terms();
int launch_qe_flush(tbpm_ctx* ctx, const RecurrenceArgs& a, int precision, const void* phi, int T, void* qe, int nE,
                    const double* coef, int n0);
int launch_qe_coefficients(tbpm_ctx* ctx, const double* table, int n_steps, int n_terms, const double* energies,
                           int nE, double H0, double tphys, double* phase, double* coef);
int launch_qe_coefficients_phase_only(tbpm_ctx* ctx, const double* energies, int nE, double tphys, int n_steps,
                                      double* phase);

// temporal fusion (csrc/fused.cu)
bool fused_applicable(const tbpm_lattice* lat, int precision, int Spad);
// register-resident sweep (variants 8-10, csrc/sweep.cu); its bounded waits report through the
// int status word at ctx->pinned + kSweepStatusSlot (zeroed at context creation)
constexpr int kSweepStatusSlot = 16;
int launch_sweep_pass(tbpm_ctx* ctx, const tbpm_lattice* lat, const RecurrenceArgs& ra, const void* prev_in,
                      const void* cur_in, void* prev_out, void* cur_out, int step0, int variant);
int sweep_status(tbpm_ctx* ctx);  // TBPM_ETIMEOUT (and clears the word) after an expired wait
// window pass of the time blocks (no moments): phi_{n+1..n+4} into win[0..3]
bool sweep_window_applicable(const tbpm_lattice* lat, int precision, int Spad);
int launch_sweep_window(tbpm_ctx* ctx, const tbpm_lattice* lat, const RecurrenceArgs& ra, const void* prev_in,
                        const void* cur_in, void* const win[4]);
int fused_steps(int variant);
int launch_fused_pass(tbpm_ctx* ctx, const tbpm_lattice* lat, const RecurrenceArgs& ra, const void* prev_in,
                      const void* cur_in, void* prev_out, void* cur_out, int step0, int variant);

enum { ACC_FIRST = 0, ACC_REGULAR = 1, ACC_NOSPMV = 2 };

// reconstruction
int launch_bessel_table(tbpm_ctx* ctx, double tau, int n_steps, int n_terms, double* table,
                        int* n_per_step);
int launch_corr_from_moments(tbpm_ctx* ctx, const double* table, const int* n_per_step, int n_steps,
                             int n_terms, const double* mu, int S, int M, double shift, double tau,
                             double* C);
int launch_dos_jackson_fp64(tbpm_ctx* ctx, const double* mu, int S, int M, const double* energies,
                            int64_t nE, double H0, double half, double* D);
int launch_dos_jackson_tensor(tbpm_ctx* ctx, const double* mu, int S, int M, const double* energies,
                              int64_t nE, double H0, double half, double* D);
// same, without synchronising: the GEMM's bounded-wait status is copied to pinned *h_err
int launch_dos_jackson_tensor_async(tbpm_ctx* ctx, const double* mu, int S, int M, const double* energies,
                                    int64_t nE, double H0, double half, double* D, int* h_err);
// electronic conductivity (csrc/conduct.cu)
void current_weights(int kind, int direction, double t, double kw[2][6]);
int launch_current(tbpm_ctx* ctx, const tbpm_lattice* lat, int precision, int S, int direction, const void* x,
                   void* y);
int launch_xdot(tbpm_ctx* ctx, int precision, int S, int64_t n_sites, const void* A, int nA, const void* B, int nB,
                double* out, int64_t os, int64_t oa, int64_t ob, int64_t off);
int launch_partial_reduce(tbpm_ctx* ctx, const double* partials, int G, int nA, int nB, int S, double* out,
                          int64_t os, int64_t oa, int64_t ob, int64_t off);
int launch_ec_corr_from_moments(tbpm_ctx* ctx, const double* table, const int* n_per_step, int n_steps,
                                const double* m, int rows, int Nn, double shift, double tau, double* C);
int launch_ec_finish(tbpm_ctx* ctx, double* C, const double* nrm, const double* energies, int nE, int rows,
                     int n_steps, double tphys, double area, double* sigma);
// Fermi-Dirac filtered responses (csrc/response.cu)
int launch_fermi_coefficients(tbpm_ctx* ctx, double mu, double kT, double H0, double half, int sqrt_f, int n_cap,
                              int K, double* scratch, double* coef);
int launch_density_phases(tbpm_ctx* ctx, const tbpm_lattice* lat, const double q[3], double2* phase);
int launch_pair_init(tbpm_ctx* ctx, int precision, int64_t n, int Sh, const void* psi, const void* opsi,
                     const double2* phase, void* xc);
int launch_pair_split(tbpm_ctx* ctx, int precision, int64_t n, int Sh, const void* psi, const void* opsi,
                      const double2* phase, void* f);
int launch_xmy(tbpm_ctx* ctx, const tbpm_lattice* lat, int precision, int Sh, int alpha, const double2* phase,
               const void* Y, int bb, size_t pair_bytes, double* C, int64_t os, int64_t off);
int launch_abs2py(tbpm_ctx* ctx, int precision, const void* Y, int bb, size_t block_bytes, int64_t n_elems,
                  double scale, double* z);
int launch_cd_finish(tbpm_ctx* ctx, const double* z, int64_t n, int S, int Spad, double factor, double* out);
int launch_oc_spectrum(tbpm_ctx* ctx, const double* C, int S, int n_steps, double dw, int n_omega, double kT,
                       double tphys, double area, int window, double* out);
int launch_dp_spectrum(tbpm_ctx* ctx, const double* C, int S, int n_steps, const double* omegas, int n_omega,
                       double tphys, double area, int window, double* out);
// FP64 D_i of a lattice (made on first use), and a request's initial state block
int lattice_ensure_d64(tbpm_lattice* lat);
int init_request_states(tbpm_ctx* ctx, const tbpm_lattice* lat, const tbpm_request* req, void* dst);
int launch_dos_fourier(tbpm_ctx* ctx, const double* C, int S, int n_steps, const double* energies,
                       int64_t nE, double tau_phys, int window, double* D);

// host-side FP64 Bessel (truncation orders, coefficient tables for the block forms)
void bessel_j_host(double x, int n_max, double* out);
int64_t truncation_order_host(double tau);

}  // namespace tbpm
