/*
 * tbpm.h -- C ABI of the GB300 (sm_103a) Chebyshev stochastic-propagation library.
 *
 * The library computes, on one GPU, the hot path of the concurrent stochastic
 * propagation method of Fu, Li, Zhou and Yuan, "Large-scale stochastic propagation
 * method beyond the sequential approach" (arXiv 2510.17432):
 *
 *   - a tight-binding Hamiltonian H on a square, honeycomb or simple-cubic lattice
 *     (nearest-neighbour hopping t, Anderson on-site disorder of width W, optional
 *     random vacancies), rescaled to H~ = (H - H0)/|H| (Sec. II.A);
 *   - blocks of S random-phase states (or site states |r> for the LDOS, Sec. III);
 *   - the Chebyshev recurrence T_{k+1} = 2 H~ T_k - T_{k-1} (App. B, Eq. cheb_relation)
 *     applied to all S states at once, fused with the inner products that give
 *     Chebyshev moments m_n = <psi|T_n(H~)|psi> (Sec. II.A, moment-based form, with the
 *     cost-halving identity of Eq. cheby_prod) or time-correlation values;
 *   - the sequential form and the state-based concurrent form with time blocks of b
 *     steps (Sec. II.A Eq. TE, Sec. II.B), both driven by Bessel coefficients
 *     c_n(tau~) = 2(-i)^n J_n(tau~) (App. B);
 *   - reconstruction of C(t_j) and of the DOS on an energy grid (Sec. III).
 *
 * Conventions shared by every entry point:
 *   - Every call returns a tbpm_status (0 = success, negative = error).  On error the
 *     thread-local message of tbpm_last_error() says what failed.  No exception
 *     crosses the ABI.
 *   - Units: hbar = 1; energies in the unit of the hopping t; times in 1/energy.
 *   - Handles (tbpm_ctx, tbpm_lattice) are created and freed by the library.  Inputs
 *     are read during the call and never retained.  Host output buffers are
 *     caller-allocated with the lengths stated per call.
 *   - Complex numbers are stored as (re, im) pairs.  Host outputs are FP64.
 *   - "_device" entry points take device pointers on the context's device and enqueue
 *     work on the context's stream without synchronising; everything else
 *     synchronises before returning.
 *   - Device memory is allocated by the library (stream-ordered) and cached in the
 *     context; it is released by tbpm_destroy().
 */
#ifndef TBPM_H
#define TBPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TBPM_OK = 0,
  TBPM_EINVAL = -1,       /* invalid argument: a message names it */
  TBPM_ENOMEM = -2,       /* device allocation failed / request exceeds the HBM budget */
  TBPM_ECUDA = -3,        /* a CUDA runtime call failed: the message carries its text */
  TBPM_ETIMEOUT = -4,     /* a bounded wait expired */
  TBPM_EUNSUPPORTED = -5, /* valid but not implemented combination */
  TBPM_EBUSY = -6,        /* serving queue full */
  TBPM_ECANCELLED = -7    /* request cancelled */
} tbpm_status;

/* lattice kinds and Hamiltonian storage paths */
enum { TBPM_SQUARE = 0, TBPM_HONEYCOMB = 1, TBPM_CUBIC = 2 };
enum { TBPM_PATH_AUTO = 0, TBPM_PATH_STENCIL = 1, TBPM_PATH_CSR = 2 };
/* state precision: complex64 states with FP64 reductions, or complex128 throughout */
enum { TBPM_C64 = 0, TBPM_C128 = 1 };
/* initial states: random phases (Sec. II.A) or site states |r> (LDOS, Sec. III) */
enum { TBPM_STATES_RANDOM = 0, TBPM_STATES_SITES = 1 };
/* propagation form (Sec. II.A): sequential, moment-based, state-based, energy-based concurrent */
enum { TBPM_SEQUENTIAL = 0, TBPM_CONCURRENT_M = 1, TBPM_CONCURRENT_S = 2, TBPM_CONCURRENT_E = 3 };
/* DOS reconstruction: Jackson-damped Chebyshev series, or windowed Fourier transform of C(t) */
enum { TBPM_DOS_JACKSON = 0, TBPM_DOS_FOURIER = 1 };
enum { TBPM_WINDOW_NONE = 0, TBPM_WINDOW_HANN = 1 };
/* reconstruction arithmetic: FP64 CUDA cores, or tensor cores (bf16x3 split, FP32 MMA, FP64 sums) */
enum { TBPM_RECON_FP64 = 0, TBPM_RECON_TENSOR = 1 };

typedef struct tbpm_ctx tbpm_ctx;
typedef struct tbpm_lattice tbpm_lattice;

/*
 * Lattice description.  Site numbering (the paper prints none; this is the library's):
 *   square     i = y*Lx + x,             neighbours (x+1,y) (x-1,y) (x,y+1) (x,y-1)
 *   honeycomb  i = 2*(y*Lx + x) + s,     A(x,y)-B(x,y), A(x,y)-B(x-1,y), A(x,y)-B(x,y-1)
 *   cubic      i = (z*Ly + y)*Lx + x,    neighbours +-x, +-y, +-z
 * H_ij = t on every bond, H_ii = V_i = W*((u>>8)*2^-24 - 1/2) with u the Philox4x32-10
 * draw (key = seed, counter = (i, 0, 0, 0) in 32-bit words (i_lo, i_hi, stream 0, 0)).
 * Vacancies (vacancy_frac > 0): site i is removed when its stream-1 draw u < floor(p*2^32);
 * the remaining sites are renumbered in order and stored on the CSR/ELL path.
 * Spectral bounds (Gershgorin; Sec. II.A uses Lanczos): E_max = max_i(V_i + deg_i|t|),
 * E_min = min_i(V_i - deg_i|t|), H0 = (E_max+E_min)/2, |H| = 1.01*(E_max-E_min)/2.
 *
 * Long-range hopping (cutoff > 0; stands in for the dense Hamiltonians of density D_H =
 * 60..230 that Sec. IV benchmarks): every site j with 0 < |r_j - r_i| <= cutoff is bonded
 * with t(r) = t exp(-(r - 1)/decay).  Distances are in units of the nearest-neighbour
 * distance; positions: square (x, y), cubic (x, y, z), honeycomb x a1 + y a2 + s (1, 0) with
 * a1 = (3/2, sqrt3/2), a2 = (3/2, -sqrt3/2).  The bonds of a site are its "taps", listed by
 * tbpm_lattice_taps(); periodic directions wrap each tap's target by modulo (a tap that
 * lands on a site another tap reaches adds to that bond; one that lands on the site itself
 * adds to the diagonal), open directions drop it.  The Gershgorin radius is the sum of |t(r)|
 * over the taps that reach active sites.  Such lattices run on the CSR/ELL path with
 * per-tap weights (path CSR), or, with path AUTO and no vacancies on square and honeycomb
 * lattices, on a matrix-free tap kernel for complex64 blocks of >= 2 states (the ELL lists are
 * then built only when another pass needs them).  In the current operator (conductivity,
 * optical conductivity) every tap carries its own bond vector.  The serving loop rejects
 * long-range lattices (TBPM_EUNSUPPORTED).
 */
typedef struct {
  int32_t kind;        /* TBPM_SQUARE / TBPM_HONEYCOMB / TBPM_CUBIC */
  int32_t path;        /* TBPM_PATH_*; AUTO picks STENCIL unless vacancy_frac > 0 */
  int64_t L[3];        /* Lx, Ly, Lz (unit cells for the honeycomb; unused entries 1) */
  int32_t pbc[3];      /* 1 = periodic, 0 = open, per direction */
  int32_t reserved;
  double t;            /* hopping */
  double W;            /* disorder width: V_i uniform on [-W/2, W/2) */
  double vacancy_frac; /* probability that a site is removed */
  uint64_t seed;       /* Philox key of the disorder and vacancy streams */
  double cutoff;       /* 0: nearest neighbours only; > 0: long-range hopping radius (<= 12) */
  double decay;        /* decay length of t(r) (> 0 when cutoff > 0) */
} tbpm_lattice_desc;

typedef struct {
  int64_t n_full;      /* sites before vacancy removal */
  int64_t n_sites;     /* active sites N (the state length) */
  int64_t n_bonds;     /* directed bonds (off-diagonal non-zeros of H) */
  int32_t path;        /* resolved TBPM_PATH_STENCIL or TBPM_PATH_CSR */
  int32_t coordination;
  double E_min, E_max; /* Gershgorin bounds */
  double H0;           /* spectral centre */
  double half_width;   /* |H| */
} tbpm_lattice_props;

/*
 * One spectral request.  S = n_states random-phase states drawn from Philox with
 * key = state_seed and counter (i_lo, i_hi, 2, s) for full site index i and state s,
 * psi_i = exp(2 pi i u/2^32)/sqrt(N); or, with states = TBPM_STATES_SITES, the S site
 * states |sites[s]> (compact site indices).
 */
typedef struct {
  int32_t precision;    /* TBPM_C64 or TBPM_C128 */
  int32_t states;       /* TBPM_STATES_RANDOM or TBPM_STATES_SITES */
  int32_t n_states;     /* S >= 1 (for SITES: the number of entries in sites) */
  int32_t form;         /* TBPM_SEQUENTIAL / TBPM_CONCURRENT_M / TBPM_CONCURRENT_S */
  uint64_t state_seed;
  const int64_t* sites; /* host array [n_states] for TBPM_STATES_SITES, else NULL */
  int64_t n_moments;    /* M (even); 0 = derive from n_steps as N(n_steps*tau~) */
  int64_t n_steps;      /* N_t time steps for correlation requests */
  double tau;           /* rescaled time step tau~; 0 means pi (the Nyquist step, Sec. II.A) */
  int32_t time_block;   /* b for TBPM_CONCURRENT_S; 0 = from the Tab. I cost model */
  int32_t dos_method;   /* TBPM_DOS_JACKSON or TBPM_DOS_FOURIER */
  int32_t window;       /* TBPM_WINDOW_* for the Fourier DOS */
  int32_t recon;        /* TBPM_RECON_FP64 or TBPM_RECON_TENSOR */
} tbpm_request;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`: a stream and a cached workspace.
 * *out receives the handle.  Fails with TBPM_ECUDA if the device is unusable. */
int tbpm_create(tbpm_ctx** out, int device);
/* Free the context and all device memory it holds.  NULL is accepted. */
int tbpm_destroy(tbpm_ctx* ctx);
/* Thread-local text of the last error (never NULL; empty after success). */
const char* tbpm_last_error(void);
/* The context's cudaStream_t, returned as void*, for event timing by the caller. */
void* tbpm_stream(tbpm_ctx* ctx);
/* Block until all work enqueued on the context's stream has finished.  Returns TBPM_ETIMEOUT
 * (once) when a bounded device wait of a fused moment pass expired since the last check; the
 * synchronous tbpm_moments and tbpm_dos report it the same way. */
int tbpm_sync(tbpm_ctx* ctx);
/* Number of kernels the library has launched on this context since creation. */
int64_t tbpm_launch_count(const tbpm_ctx* ctx);
/* Temporal fusion of the moment pass (several Chebyshev steps per pass, so each state vector
 * crosses HBM twice per pass instead of three times per step), used where a fused kernel exists
 * (honeycomb stencil, complex64, S >= 2, lattice at least 48 x 32 cells).
 * mode: 0 = one step per pass; 1 = 4 steps per pass (2-D tiles); 2 = 2 steps per pass (2-D tiles);
 * 3, 4 = 2 steps per pass by a row sweep (bands of cells, rows of phi_n streamed through a
 * shared-memory ring one row ahead, each further step one row behind the previous; 128- and
 * 256-thread CTAs); 5, 6 = the row sweep with 4 steps per pass (128- and 256-thread CTAs);
 * 7 = the 2-step sweep in the same code as 5 and 6; 8, 9, 10 = 4 steps per pass by a
 * register-resident sweep (each thread keeps the recurrence levels of its cell in registers and
 * exchanges only the x-neighbours through shared memory, one barrier per row; rows of phi_n and
 * phi_{n-1} arrive by TMA bulk copies; 128-, 192- and 256-thread CTAs; a lattice narrower than
 * one band takes mode 5).  Default 8.  -1 = the fastest of modes 0, 4, 5 and 8 timed on the
 * request's lattice shape.  Results of different modes agree within the complex64 tolerance, not
 * bit for bit; each mode is deterministic.  Modes outside -1..10 are rejected with TBPM_EINVAL. */
int tbpm_set_fusion(tbpm_ctx* ctx, int mode);
/* mode -1 = autotuned: the first moment request on a lattice shape (kind, sizes, boundaries,
 * path, padded S, precision, disorder) with at least 128 moments times 24 steps of each of modes
 * 0, 4, 5 and 8 on scratch buffers and keeps the fastest for that shape in the context.  Results
 * of different modes agree within the complex64 tolerance, not bit for bit.
 * tbpm_fusion_report: ms per step of each mode in the last autotune (index = mode 0..15, -1 = not
 * timed); the caller's array holds 16 doubles. */
int tbpm_fusion_report(tbpm_ctx* ctx, double ms_per_step[16]);
/* CUDA graphs for the moment pass (default on): a moment request whose pass sequence (buffers,
 * lattice, sizes, fusion mode) repeats a previous one is captured into a CUDA graph on its
 * second occurrence and replayed from the third on, so a small lattice no longer pays one host
 * launch per Chebyshev step.  Results are bit-identical with graphs on or off.  Phase timing
 * (tbpm_profile) runs the passes without graphs.  enable = 0 drops the cached graphs. */
int tbpm_set_graphs(tbpm_ctx* ctx, int enable);
/* Buffered time blocks (default on): the state-based and sequential forms (Sec. II.B, Eq. TE)
 * keep the Chebyshev vectors phi_n of up to 32 consecutive terms in buffer slots and add
 * sum_n c_n(j tau~) phi_n to every open accumulator of the block in one pass, instead of one
 * accumulator update per term; C(t_j) = <psi|psi(t_j)> of the block then comes from one block
 * inner product.  The arithmetic is the same sum in another order (results agree to rounding).
 * The buffer takes up to 34 state blocks and shrinks with free memory; with fewer than 4 slots,
 * the sequential form (b = 1), or enable = 0, every term updates the accumulators in the
 * recurrence pass itself. */
int tbpm_set_block_buffering(tbpm_ctx* ctx, int enable);
/* Memory control of the Fermi-Dirac filtered quantities (tbpm_optical_conductivity,
 * tbpm_polarization, tbpm_charge_density): their states are processed in passes of at most
 * max_states states (rounded down to a power of two; 0 = as many as fit in 85% of the free device
 * memory, at most 16).  A pass holds at most three pair blocks (2 x its states) during the
 * Fermi-Dirac series and 2 + b during the propagation; results do not depend on the pass width.
 * No counterpart in the paper (its states fit in host memory). */
int tbpm_set_pass_states(tbpm_ctx* ctx, int max_states);
/* Phase timing.  tbpm_profile(ctx, 1) clears the record and starts recording CUDA events
 * on the context stream around every recurrence loop of a moment request (kind 0: all its
 * passes), around its fused multi-step passes (kind 2, a sub-interval of kind 0) and around
 * every DOS reconstruction (kind 1); tbpm_profile(ctx, 0) stops.  tbpm_profile_read()
 * synchronises and returns, summed over the recorded phases: out[0] = recurrence ms,
 * out[1] = recurrence kernel launches, out[2] = reconstruction ms, out[3] = reconstruction
 * launches, out[4] = fused-pass ms, out[5] = fused-pass launches. */
int tbpm_profile(tbpm_ctx* ctx, int enable);
int tbpm_profile_read(tbpm_ctx* ctx, double out[6]);

/* ---------------------------------------------------------------- lattice */

/* Build H on the device: disorder, vacancies, CSR/ELL neighbour lists and bounds.
 * The lattice stays valid until tbpm_lattice_destroy() and must be destroyed before
 * its context.  Sizes: every L >= 1, product of sites < 2^31 * 2 (see n_sites). */
int tbpm_lattice_create(tbpm_ctx* ctx, const tbpm_lattice_desc* desc, tbpm_lattice** out);
int tbpm_lattice_destroy(tbpm_lattice* lat);
int tbpm_lattice_info(const tbpm_lattice* lat, tbpm_lattice_props* out);
/* Debug export for bit-exact tests (any pointer may be NULL):
 *   compact  [n_full]        compact index of every full site, -1 if vacant
 *   V        [n_sites]       FP64 on-site energies
 *   nbr      [n_sites * z]   neighbour compact indices in the fixed order, -1 if none */
int tbpm_lattice_export(const tbpm_lattice* lat, int64_t* compact, double* V, int32_t* nbr);
/* Taps of the lattice, one per neighbour slot of the ELL lists (any pointer may be NULL):
 *   offsets [z][4]  (dx, dy, dz, ds): a site of sublattice 0 (every site of the square and
 *                   cubic lattices) in cell (x,y,z) reaches cell (x+dx, y+dy, z+dz) of
 *                   sublattice ds; a honeycomb B site reaches (x-dx, y-dy) of sublattice 1-ds
 *   t       [z]     hopping of the slot, t(r) (t itself on nearest-neighbour lattices)
 * z = tbpm_lattice_props.coordination.  Nearest-neighbour lattices report their fixed order. */
int tbpm_lattice_taps(const tbpm_lattice* lat, int32_t* offsets, double* t);

/* Which kernel carries the moment recurrence (a4) of a request on this lattice under the
 * context's fusion mode (a diagnostic for benchmarks and profiles; no device work):
 *   TBPM_PASS_STENCIL  one-step matrix-free stencil pass (k_moment_stencil)
 *   TBPM_PASS_ELL      one-step pass over ELL neighbour lists (vacancies; k_moment_step)
 *   TBPM_PASS_TAPS     matrix-free tap kernel of a long-range lattice (k_taps_moment)
 *   TBPM_PASS_SWEEP    four-step register sweep (fusion modes 8-10; k_sweep_moments)
 *   TBPM_PASS_ROWS     row-sweep fused pass with shared-memory level rings (modes 3-7)
 *   TBPM_PASS_TILES    2-D tile fused pass (modes 1, 2)
 * Under fusion mode -1 a fused lattice reports TBPM_PASS_STENCIL (the mode is chosen by timing
 * at the first request).  Errors: TBPM_EINVAL for NULL arguments or an invalid request. */
/* Index checks of a debug build (libtbpm_debug.so, compiled with TBPM_DEBUG; the paper has no
 * counterpart).  There the hot kernels (stencil, ELL and serving passes, the register sweep's
 * stores and row copies) skip any global-memory access whose index falls outside its buffer and
 * record the first such index per source unit; they never trap, so the context stays usable.
 * words[k] (k = 0: recurrence passes, 1: register sweep, 2: serving) = (kernel id << 48) |
 * (index & 0xFFFFFFFFFFFF), 0 when no check failed; kernel ids: 1 stencil units, 2 ELL
 * neighbour index, 3 sweep store, 4 sweep row copy, 5 serving units.  Reading clears the words
 * and synchronises the device.  The regular library returns TBPM_EUNSUPPORTED and zero words. */
int tbpm_debug_status(tbpm_ctx* ctx, uint64_t words[3]);

/* Expiry check of the device-side bounded waits (failure detection; the paper has no
 * counterpart).  The kernels fed by TMA copies (the register sweep, the tensor-core GEMM) wait
 * on mbarriers for at most 2 s each; on expiry they record a code in a status word, wait
 * (bounded) for their own copies in flight and return, so the context stays usable and the call
 * reports TBPM_ETIMEOUT.  This call runs the register sweep's bounded wait in a one-warp kernel
 * on the context stream and reports it through the sweep's status word:
 *   arrive != 0   the barrier's one expected arrival happens first; returns TBPM_OK;
 *   arrive == 0   nothing arrives and no copy is in flight; the wait gives up after budget_s
 *                 seconds and the call returns TBPM_ETIMEOUT (the status word is cleared).
 * Synchronises the context stream.  Errors: TBPM_EINVAL for a NULL context or a budget outside
 * (0, 2] seconds. */
int tbpm_wait_probe(tbpm_ctx* ctx, int arrive, double budget_s);

/* Measured FP32 FMA throughput of the context's device in TFLOP/s (an FMA counts as two flops),
 * scalar FMAs and packed f32x2 FMAs: the denominator of the roofline of the FP32-issue-bound tap
 * kernel (the paper has no counterpart; it reports CPU times).  Runs about a millisecond of
 * FMA chains on the context stream and synchronises it. */
int tbpm_fp32_fma_peak(tbpm_ctx* ctx, double* tflops_scalar, double* tflops_packed);

enum { TBPM_PASS_STENCIL = 0, TBPM_PASS_ELL = 1, TBPM_PASS_TAPS = 2, TBPM_PASS_SWEEP = 3, TBPM_PASS_ROWS = 4,
       TBPM_PASS_TILES = 5 };
int tbpm_moment_pass_kind(tbpm_ctx* ctx, const tbpm_lattice* lat, const tbpm_request* req, int* kind);

/* ---------------------------------------------------------------- states */

/* Initial state block as stored for the recurrence, exported to the host:
 * out = [S][n_sites] complex, FP64 pairs (C128) or FP32 pairs (C64).
 * draws (optional) = [S][n_sites] uint32 Philox phase draws (random states only). */
int tbpm_states_export(tbpm_ctx* ctx, const tbpm_lattice* lat, const tbpm_request* req,
                       void* out, uint32_t* draws);

/* Adjacency operator y_i = sum over the neighbours j of i of x_j, applied by the same
 * recurrence kernel as the hot path (first-term mode, zero diagonal, unit hopping).
 * x, y = host [n_sites][S] interleaved complex (FP32 pairs for C64, FP64 for C128);
 * S must be a power of two <= 32.  For exact tests of the stencil and ELL indexing. */
int tbpm_apply_hopping(tbpm_ctx* ctx, const tbpm_lattice* lat, int precision, int n_states,
                       const void* x, void* y);

/* ---------------------------------------------------------------- hot path */

/* Chebyshev moments m_n = <psi_s|T_n(H~)|psi_s>, n = 0..M-1, of every state s, from
 * M/2 matrix applications (cost-halving identity Eq. cheby_prod, with
 * m_{2k} = 2<phi_k|phi_k> - m_0 and m_{2k+1} = 2<phi_{k+1}|phi_k> - m_1).
 * mu = host [S][M][2] (re, im).  M must be even and >= 2. */
int tbpm_moments(tbpm_ctx* ctx, const tbpm_lattice* lat, const tbpm_request* req, double* mu);
/* Same, into device memory d_mu [S][M][2] doubles; asynchronous on the context stream. */
int tbpm_moments_device(tbpm_ctx* ctx, const tbpm_lattice* lat, const tbpm_request* req,
                        double* d_mu);

/* Correlation C_s(t_j) = <psi_s|exp(-i H t_j)|psi_s>, t_j = j*tau~/|H|, j = 0..N_t, by the
 * request's form: SEQUENTIAL (step by step), CONCURRENT_M (moments, then
 * C(t_j) = exp(-i H0 t_j) sum_{n<N(j tau~)} c_n(j tau~) m_n), or CONCURRENT_S (time blocks
 * of b steps, Eq. TE).  C = host [S][N_t+1][2]. */
int tbpm_correlation(tbpm_ctx* ctx, const tbpm_lattice* lat, const tbpm_request* req, double* C);
int tbpm_correlation_device(tbpm_ctx* ctx, const tbpm_lattice* lat, const tbpm_request* req,
                            double* d_C);

/* DOS (or LDOS for site states) of every state on the energies [n_energies] (host):
 *   TBPM_DOS_JACKSON: D(E) = [g_0 m_0 + 2 sum_{n>=1} g_n Re m_n T_n(E~)] / (pi |H| sqrt(1-E~^2))
 *     with Jackson factors g_n (Weisse et al., Rev. Mod. Phys. 78, 275 (2006), Eq. 71);
 *   TBPM_DOS_FOURIER: D(E) = (tau/2pi)[w_0 C(0) + 2 Re sum_j w_j exp(i E t_j) C(t_j)] (Sec. III).
 * D = host [S][n_energies].  Energies outside (H0-|H|, H0+|H|) give 0 for Jackson. */
int tbpm_dos(tbpm_ctx* ctx, const tbpm_lattice* lat, const tbpm_request* req,
             const double* energies, int64_t n_energies, double* D);
/* Same with device energies [n_energies] and device output [S][n_energies]; async. */
int tbpm_dos_device(tbpm_ctx* ctx, const tbpm_lattice* lat, const tbpm_request* req,
                    const double* d_energies, int64_t n_energies, double* d_D);

/* ---------------------------------------------------------------- serving */

/* Continuous batching of DOS / LDOS requests (moment-based form, Jackson reconstruction).
 * A scheduler thread admits queued requests in arrival order while their HBM footprint fits
 * the budget, keeps their states resident, and advances every admitted request by one
 * Chebyshev step per launch of one batched kernel -- requests of any lattice kind, size,
 * state count and moment count share each launch; requests that arrive while others run join
 * at the next launch.  Each request's tiling and reduction order depend only on its own
 * geometry, so its moments and DOS are bit-identical alone and in any mix. */
typedef struct tbpm_server tbpm_server;
typedef struct {
  size_t hbm_budget_bytes; /* device memory for resident requests; 0 = 70% of free memory */
  int32_t max_active;      /* requests advanced together; 0 = 64 */
  int32_t max_queue;       /* queued requests before tbpm_submit returns TBPM_EBUSY; 0 = 4096 */
  int32_t recon;           /* TBPM_RECON_FP64 or TBPM_RECON_TENSOR for the DOS */
  int32_t reserved;
} tbpm_server_config;

/* Start a server on ctx's device (it creates its own streams; ctx only names the device). */
int tbpm_server_create(tbpm_ctx* ctx, const tbpm_server_config* cfg, tbpm_server** out);
/* Stop the scheduler; queued and running requests end with TBPM_ECANCELLED. */
int tbpm_server_destroy(tbpm_server* srv);
/* Queue one request: lattice, request (form ignored: moment-based; n_moments even >= 2;
 * random states or site states) and the energies [n_energies].  Everything is copied.
 * *ticket identifies the request.  TBPM_EBUSY when the queue is full. */
int tbpm_submit(tbpm_server* srv, const tbpm_lattice_desc* lat, const tbpm_request* req,
                const double* energies, int64_t n_energies, uint64_t* ticket);
/* Wait up to timeout_us (< 0: forever) for a request; on success copies its DOS, [S][n_energies]
 * (D_len values available), and latency_us[3] = {queued, admitted-to-done, submit-to-done}.
 * Returns the request's status (TBPM_ETIMEOUT if not finished in time; the ticket stays valid). */
int tbpm_wait(tbpm_server* srv, uint64_t ticket, int64_t timeout_us, double* D, size_t D_len,
              double* latency_us);
/* out = {queued, active, completed, batched kernel launches, bytes reserved, byte budget,
 * device microseconds spent in the batched launches (summed over launches known complete)}. */
int tbpm_server_stats(tbpm_server* srv, int64_t out[7]);

/* ---------------------------------------------------------------- allocation-free step */

/* One pass of the moment kernel with no device allocation at all.  The paper has no
 * counterpart: this entry point exists for callers that cannot let a library allocate
 * device memory -- applications that reserve nearly all HBM in their own arena, loops
 * where a cudaMalloc/cudaFree could synchronise the device, plugin hosts that only hand
 * out buffers.  Every buffer is the caller's; the only scratch (per-block partial sums
 * and a completion counter) lives in a fixed 1 MiB __device__ array inside the library,
 * which every GPU that loads the library holds until the process exits.
 *
 * Matrix-free stencil lattices only (no vacancies).  Arguments:
 *   kind, L, pbc        lattice as in tbpm_lattice_desc; L[2] and pbc[2] are read only for
 *                       the cubic lattice, so 2-D callers may pass two-entry arrays
 *   t_scaled            t / |H|
 *   d_diag              device [N] rescaled on-site terms (V_i - H0)/|H| (float for C64,
 *                       double for C128), or NULL to use diag_const for every site
 *   precision, n_states C64 or C128; S a power of two <= 32
 *   d_cur               device phi_n, [N][S] interleaved complex
 *   d_prev_out          device phi_{n-1} on input (ignored when step == 0), phi_{n+1} on output
 *   d_mu                device [S][n_moments][2]: step 0 writes m_0, m_1; step k >= 1 writes
 *                       m_{2k} = 2<phi_k|phi_k> - m_0 and m_{2k+1} = 2<phi_{k+1}|phi_k> - m_1,
 *                       reading m_0 and m_1 back from d_mu
 *   step                k, 0 <= k < n_moments/2; stream = cudaStream_t or NULL
 * Runs on the current device and returns without synchronising.  The first call on a device
 * looks up the scratch array's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture.  All calls share the one scratch array and every call resets
 * its counter, so calls that overlap on the GPU (other streams, other host threads) race and
 * must be serialised by the caller.  Sizes whose partial sums cannot fit the scratch are
 * rejected with TBPM_EINVAL. */
int tbpm_moment_step_noalloc(int kind, const int64_t L[3], const int32_t pbc[3], double t_scaled,
                             double diag_const, const void* d_diag, int precision, int n_states,
                             const void* d_cur, void* d_prev_out, double* d_mu, int64_t n_moments,
                             int64_t step, void* stream);

/* Quasi-eigenstates (Sec. IV, Eq. QE): |Psi(E)> = (1/2pi) int e^{iEt}|psi(t)> dt, sampled at
 * t_j = j tau~/|H|, j = -N_t..N_t, for every state and energy, by the request's form:
 *   SEQUENTIAL    forward and backward step-by-step propagation (Eq. form1_sequential),
 *   CONCURRENT_S  the same states from time blocks of b steps (Eq. TE; b = 0: autotuned),
 *   CONCURRENT_E  one recurrence, |Psi(E)> = sum_n C_n(E) T_n(H~)|psi> (Eqs. form2_concurrent,
 *                 QE_coeff; C_n carries the 1/2pi of Eq. QE and exp(+-i H0 t)).
 * out = host [n_energies][S][n_sites] complex (FP32 pairs for C64, FP64 for C128).
 * Device memory: n_energies accumulating state blocks. */
int tbpm_quasi_eigenstates(tbpm_ctx* ctx, const tbpm_lattice* lat, const tbpm_request* req,
                           const double* energies, int64_t n_energies, void* out);

/* DC (electronic) conductivity (Sec. V, Eqs. DC, dc_corr, dc_mom) along `direction`
 * (0 = x, 1 = y, 2 = z for the cubic lattice), hbar = e = 1:
 *   J_a = i[H, P_a], (J_a)_ij = -i t (r_j - r_i)_a on every bond (nearest image across periodic
 *     boundaries).  Bond vectors: unit square / cubic lattices; graphene with C-C distance 1,
 *     A -> B bonds (1,0), (-1/2,-sqrt3/2), (-1/2,sqrt3/2) in the neighbour order of
 *     tbpm_lattice_export, B -> A their negatives.
 *   C(t_j, E) = <psi| J e^{iHt_j} J |Psi(E)> / |<psi|Psi(E)>|, t_j = j tau~/|H|, j = 0..N_t, with
 *     |Psi(E)> the quasi-eigenstates of tbpm_quasi_eigenstates (energy-based form for
 *     n_energies <= 200, state-based otherwise), by the request's form:
 *       SEQUENTIAL    e^{-iHt} J|psi> step by step, one inner product per step and energy,
 *       CONCURRENT_S  the same states from time blocks of b steps (b = 0: autotuned); each
 *                     block's b states meet all energies in one pass,
 *       CONCURRENT_M  moments m_n(E) = <J psi|T_n(H~)|J Psi(E)>, n < N(N_t tau~), then
 *                     C = e^{i H0 t} sum_n c_n^*(t~) m_n / |<psi|Psi(E)>|.
 *   sigma(E) = D(E)/A int_0^{N_t tau} Re[e^{-iEt} C(t,E)] dt, trapezoid weights on t_j,
 *     D(E) = N Re<psi|Psi(E)>, A = N x area per site (1; 3 sqrt3/4 for graphene).
 * C (optional, may be NULL) = host [S][n_energies][N_t+1][2]; sigma = host [S][n_energies].
 * A state whose <psi|Psi(E)> is exactly 0 gets C = 0 and sigma = 0 at that energy.
 * Errors: TBPM_EINVAL for a direction outside the lattice's dimensions, another form,
 * n_steps outside [1, 2^20], n_energies outside [1, 4096] or n_energies x S > 65536.
 * Device memory: n_energies + 4 state blocks (+ b for CONCURRENT_S). */
int tbpm_conductivity(tbpm_ctx* ctx, const tbpm_lattice* lat, const tbpm_request* req, int direction,
                      const double* energies, int64_t n_energies, double* C, double* sigma);

/* tbpm_conductivity that also returns the overlaps that normalise C: overlap (may be NULL) =
 * host [S][n_energies][2], <psi|Psi(E)> of every state and energy exactly as the device computed
 * and used it, so that C(t,E) x |<psi|Psi(E)>| recovers the un-normalised correlation
 * <J psi(t)|J Psi(E)> of Eq. dc_corr.  Same arguments, errors and device memory otherwise. */
int tbpm_conductivity_overlap(tbpm_ctx* ctx, const tbpm_lattice* lat, const tbpm_request* req, int direction,
                              const double* energies, int64_t n_energies, double* C, double* sigma,
                              double* overlap);

/* Fermi-Dirac operator (the operators f(H), f^{1/2}(H) of the OC, DP and CD sections), hbar = k_B = 1:
 *   f(E) = 1/(1 + e^{(E - mu)/kT}); out = f(H) psi (sqrt_f = 0) or f(H)^{1/2} psi (sqrt_f != 0) for
 *   the request's states, as the Chebyshev series sum_n a_n T_n(H~) psi with
 *   a_n = ((2 - delta_n0)/K) sum_k f(H0 + |H| cos th_k) cos(n th_k), th_k = pi (k + 1/2)/K
 *   (Chebyshev-Gauss quadrature), truncated at 1 + max{n : |a_n| > 1e-14} within
 *   min(2^14, 12 |H|/kT + 64) orders (kT well below |H|/1300 is therefore not resolved).
 * out = host [S][n_sites] complex (FP32 pairs for C64, FP64 for C128).
 * Errors: TBPM_EINVAL for kT <= 0 or a non-finite mu. */
int tbpm_fermi_apply(tbpm_ctx* ctx, const tbpm_lattice* lat, const tbpm_request* req, double mu, double kT,
                     int sqrt_f, void* out);

/* Optical conductivity (OC section, Eq. oc_corr and the Kubo and Kramers-Kronig relations there):
 *   C(t_j) = <psi_1(t_j)| J_alpha |psi_2(t_j)>, psi_1(t) = e^{-iHt} f(H) psi,
 *   psi_2(t) = e^{-iHt} [1 - f(H)] J_beta psi, t_j = j tau~/|H| (tau~ = pi/2 when req->tau = 0),
 *   j = 0..N_t; both states advance in one state block of 2 x pow2(S) states, by the request's
 *   form SEQUENTIAL (b = 1) or CONCURRENT_S (time blocks of b = time_block steps, 0 = autotuned).
 *   Re sigma(w_k) = 2 (e^{-w_k/kT} - 1)/(w_k a) tau sum_j w_j sin(w_k t_j) Im C(t_j), w_k = k w_max/(n_omega-1),
 *   w_j = window_j (2 - delta_j0)/2, a = area per site (1; 3 sqrt3/4 for graphene; the sample's
 *   trace N C over its area N a); Re sigma(0) = 0 (no Drude term).
 *   Im sigma(w_k) = -(2 w_k/pi) sum_{j: j-k odd} Re sigma(w_j) c_j/(w_j^2 - w_k^2), c_0 = dw, c_j = 2 dw
 *   (Kramers-Kronig, principal value by Maclaurin's rule).
 * C (optional, may be NULL) = host [S][N_t+1][2]; sigma = host [S][n_omega][2] (Re, Im).
 * Any S <= 32: the states run in passes of at most 16 (fewer when memory is short, see
 * tbpm_set_pass_states).
 * Errors: TBPM_EINVAL for directions outside the lattice's dimensions, kT <= 0, another form,
 * n_steps outside [1, 2^22], n_omega outside [2, 2^20] or w_max <= 0; TBPM_ENOMEM when not even
 * one state's pass fits. */
int tbpm_optical_conductivity(tbpm_ctx* ctx, const tbpm_lattice* lat, const tbpm_request* req, int alpha,
                              int beta, double mu, double kT, double omega_max, int64_t n_omega, double* C,
                              double* sigma);

/* Dynamical polarization (DP section): C(t_j, q) = <psi_1(t_j)| rho(q) |psi_2(q, t_j)>,
 *   rho(q) = sum_i e^{i q.r_i}|i><i|, psi_1 as for the OC, psi_2(q, t) = e^{-iHt} [1 - f(H)] rho(-q) psi;
 *   Pi(q, w) = -(2/a) tau sum_j w_j e^{i w t_j} Im C(t_j, q) for each caller-given w.
 *   Site positions r_i: unit square / cubic lattices at (x, y, z); graphene A(x,y) = x a1 + y a2,
 *   B(x,y) = A(x,y) + (1, 0), a1 = (3/2, sqrt3/2), a2 = (3/2, -sqrt3/2).
 * q = host [3]; C (optional) = host [S][N_t+1][2]; Pi = host [S][n_omega][2] (Re, Im).
 * Errors as for tbpm_optical_conductivity (n_omega in [1, 2^20]). */
int tbpm_polarization(tbpm_ctx* ctx, const tbpm_lattice* lat, const tbpm_request* req, const double q[3],
                      double mu, double kT, const double* omegas, int64_t n_omega, double* C, double* Pi);

/* Charge density (CD section, Eq. rho), read as N times the weighted time average of the integrand
 * over the sampled window (the integrand of a finite sample does not decay):
 *   rho_i = N sum_{j=0}^{N_t} w_j |psi(t_j)_i|^2 / sum_j w_j,  psi(t) = e^{-iHt} f^{1/2}(H) psi,
 *   w_j = (2 - delta_j0)/2, t_j = j tau~/|H|; req->tau = 0 selects tau~ = pi |H| / Delta_occ with
 *   Delta_occ = min(E_max, mu + 20 kT) - E_min (the integrand's band is 2 Delta_occ wide).
 *   Forms SEQUENTIAL (b = 1) or CONCURRENT_S (b = time_block, 0 = autotuned); abs2py
 *   (z_i += |x_i|^2) runs once per time block over all of its states.  N_t = 0 gives the plain
 *   estimate N |<i|f^{1/2}|psi>|^2.
 * rho = host [S][n_sites] (FP64).  Errors: TBPM_EINVAL for kT <= 0, mu below the spectrum,
 * n_steps outside [0, 2^22] or another form. */
int tbpm_charge_density(tbpm_ctx* ctx, const tbpm_lattice* lat, const tbpm_request* req, double mu, double kT,
                        double* rho);

/* ---------------------------------------------------------------- cost model */

/* Truncation order N(tau~) = 1 + max{n : |c_n(tau~)| > 1e-14} (Sec. II.A), FP64 host. */
int64_t tbpm_truncation_order(double tau);
/* Tab. I counts of the state-based form with blocks of b steps over N_t steps:
 * out[0] = amxsy (Chebyshev terms generated), out[1] = axpy, out[2] = dot. */
int tbpm_block_counts(int64_t n_steps, int64_t b, double tau, int64_t out[3]);
/* b_opt = argmin_b N_amxsy(b) t_amxsy + N_axpy(b) t_axpy over 1 <= b <= b_max (Sec. II.B). */
int64_t tbpm_block_opt(int64_t n_steps, double tau, double t_amxsy, double t_axpy, int64_t b_max);
/* Autotuner of the state-based form (Sec. II.B: the per-operation costs are "obtained via
 * benchmarking prior to the main calculation"): times recurrence passes with no and with
 * several open accumulators on this lattice and request (precision, S), then returns
 * *b_opt = tbpm_block_opt(...) with b capped by the free device memory (and by 256).
 * times_ms (optional) receives t_amxsy and t_axpy in milliseconds.  CONCURRENT_S requests
 * with time_block = 0 use it. */
int tbpm_block_autotune(tbpm_ctx* ctx, const tbpm_lattice* lat, const tbpm_request* req, int64_t n_steps,
                        int64_t* b_opt, double times_ms[2]);

#ifdef __cplusplus
}
#endif
#endif /* TBPM_H */
