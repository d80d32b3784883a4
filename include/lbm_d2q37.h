/*
 * lbm_d2q37.h - C ABI of the GB300 (sm_103a) D2Q37 thermal lattice-Boltzmann step.
 *
 * Method: arXiv:1703.04594 (Calore, Gabbana, Schifano, Tripiccione), Sec. 3.
 *   One time step is  propagate -> bc -> collide  (Sec. 5, kernel sequence):
 *   - propagate (pull form, eq. "master2"): f~_i(x, y) = f_i(x - v_i, t), 37 populations
 *     hopping up to three sites (Fig. "streamscheme"); x is periodic.
 *   - bc: thermal walls at y = 0 and y = Ly - 1 act on the three outermost rows (Sec. 5).
 *     A population pulled from outside the fluid takes the wall equilibrium
 *     f_i^eq(rho_w, 0, T_wall), rho_w = density at the start of the step of the fluid site
 *     next to the wall in the source column.
 *   - collide: BGK relaxation (eq. "lbequation") towards the fourth-order Hermite
 *     equilibrium of the moments (eq. "macro"), evaluated at the gravity-shifted velocity
 *     u + tau g and temperature T + tau (1 - tau) |g|^2 / D.
 *
 * Units: molecular velocities xi_i = c v_i with integer hops v_i and the lattice scale c
 * (see lbm_model); velocity, temperature and gravity are in xi units, reference T0 = 1.
 *
 * Layout (structure of arrays, Sec. 4, "SoA"; y contiguous, two copies read and written
 * alternately): population i of site (x, y) is element  i*lx*pitch + x*pitch + y  of a
 * state buffer.  pitch = lbm_pitch(p) >= ly; elements y >= ly of a column are padding and
 * are never read.  FP64 and FP64_FIXED states hold double f_i.  FP32_SHIFTED and FP32_CONSERVED states hold float
 * (f_i - w_i * rho0).  Population order: 0 = rest, 1..18 = the vectors returned by
 * lbm_model in that order, 18 + k = -(vector k).
 *
 * Conventions for every call:
 *   - Pointers named *_dev are device pointers; *_host are host pointers.  The caller
 *     owns every buffer and the stream; no entry point allocates device memory except
 *     lbm_batch_plan (its tables, freed by lbm_batch_destroy) and lbm_probe_peak (a result
 *     buffer it frees before returning).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls
 *     are stream-ordered and asynchronous unless stated otherwise.
 *   - Return value: LBM_OK, or an lbm_status error code.  Invalid arguments are
 *     rejected with LBM_EINVAL before anything is launched.  LBM_ECUDA reports a launch
 *     or copy failure; lbm_last_cuda_error() returns the CUDA error code.
 *   - State buffers must be 16-byte aligned (cudaMalloc and torch give 256); a
 *     step's input and output must not overlap (the pull scheme needs two copies).
 */
#ifndef LBM_D2Q37_H
#define LBM_D2Q37_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum lbm_status { LBM_OK = 0, LBM_EINVAL = 1, LBM_ECUDA = 2, LBM_ETIMEOUT = 3, LBM_ENOMEM = 4, LBM_ESIZE = 5 };
/* LBM_FP64: float64 populations, float64 collision arithmetic (moment sums in exact 64-bit
 * fixed point for sites whose populations are all below 8 in magnitude, plain float64 sums
 * for any other site, so every finite state is handled; a non-finite population makes its
 * site's outputs NaN; the sums' conversion and the products by powers of two run on the
 * integer pipe, with the bits of their float64 counterparts).  LBM_FP32_SHIFTED: float32 storage of g_i = f_i - w_i rho0, for
 * states with every |g_i| < 8 (choose rho0 near the state's density); a site holding a
 * larger deviation, an infinity or a NaN gets NaN moments, and every population it
 * produces is NaN.  LBM_FP64_FIXED:
 * float64 populations as LBM_FP64 (same buffers, interchangeable states); the fused step
 * evaluates the equilibrium polynomial and the relaxation of every population in 64-bit
 * fixed point on the integer pipes, with errors below one float64 rounding unit, for sites
 * in a stated physical range (float64 elsewhere).  lbm_step, lbm_run, lbm_init, lbm_moments,
 * lbm_kinetic_energy*, lbm_simulate_host and the batch entry points accept it; the separate
 * kernels, layouts and adjoint entry points take LBM_FP64 (its states are the same). */
/* LBM_FP32_CONSERVED: the FP32_SHIFTED storage (same buffers, interchangeable states) with a
 * collision that restores the exact post-collision mass, momentum and energy of every site
 * after its float32 arithmetic (a second, exact moment sum over the outputs and a correction
 * along w_i (alpha + beta . v_i + gamma (|v_i|^2 - m)), the first Hermite polynomials over all
 * 37 populations): float32 rounding then no longer accumulates in the conserved fields,
 * which is what limits the velocity accuracy of long FP32_SHIFTED runs.  Accepted wherever
 * LBM_FP32_SHIFTED is. */
enum lbm_precision { LBM_FP64 = 0, LBM_FP32_SHIFTED = 1, LBM_FP64_FIXED = 2, LBM_FP32_CONSERVED = 3 };
enum lbm_bc { LBM_BC_WALLS = 0, LBM_BC_PERIODIC_Y = 1 /* test mode: y wraps like x */ };

/* Problem parameters, as the paper states the problem (Sec. 3): lattice size, BGK
 * relaxation time tau (> 0.5), gravity (gx, gy) per time step in xi units, wall
 * temperatures.  rho0 is the reference density of the FP32_SHIFTED storage.
 * Constraints: lx >= 4, ly >= 6, lx * lbm_pitch < 2^32, lx <= 262140. */
typedef struct lbm_params {
  int32_t lx, ly;
  int32_t precision; /* enum lbm_precision */
  int32_t bc;        /* enum lbm_bc */
  double tau;
  double gx, gy;
  double t_bottom, t_top;
  double rho0;
} lbm_params;

/* Library ABI version (incremented on any incompatible change). */
int32_t lbm_version(void);

/* Model constants (host only, no GPU needed): lattice scale c, the 37 weights w_i and
 * integer hops (vx_i, vy_i) in the library's population order.  Any pointer may be NULL.
 * Sec. 3 / Fig. "streamscheme" for the 37 hops; the weights and c solve the lattice
 * isotropy conditions up to eighth order. */
int32_t lbm_model(double* c, double* w37, int32_t* vx37, int32_t* vy37);

/* Elements per y-column of a state buffer (ly rounded up to 32), or -1 if p is invalid. */
int64_t lbm_pitch(const lbm_params* p);
/* Bytes of one state buffer: 37 * lx * pitch * element size, or -1 if p is invalid. */
int64_t lbm_buffer_bytes(const lbm_params* p);

/* Populations at local equilibrium with the given fields (Sec. 3: an LB run starts from
 * an assignment of the populations matching the initial condition):
 * f_i = f_i^eq(rho, (ux, uy), T).  Fields are [lx][ly] doubles, y contiguous. */
int32_t lbm_init(const lbm_params* p, const double* rho_dev, const double* ux_dev,
                 const double* uy_dev, const double* T_dev, void* f_dev, void* stream);

/* One fused time step (propagate + bc + collide in a single pull kernel):
 * f_out = step(f_in).  f_in and f_out must not overlap. */
int32_t lbm_step(const lbm_params* p, const void* f_in_dev, void* f_out_dev, void* stream);

/* n_steps fused steps, alternating between the two buffers (the paper's two lattice
 * copies, Sec. 4).  The result is in f_a when n_steps is even, else in f_b. */
int32_t lbm_run(const lbm_params* p, void* f_a_dev, void* f_b_dev, int32_t n_steps, void* stream);

/* The step as three separate kernels, in the paper's order (Sec. 5):
 *   lbm_propagate: f_tmp_i(x, y) = f_in_i(x - vx_i, y - vy_i) for every source inside
 *                  the fluid (entries whose source is outside are left untouched);
 *   lbm_bc:        writes the wall equilibria into exactly those entries of f_tmp, with
 *                  rho_w taken from f_in;
 *   lbm_collide:   f_out = collide(f_tmp), site by site.
 * propagate -> bc -> collide equals lbm_step up to floating-point contraction order.
 * FP64 only. */
int32_t lbm_propagate(const lbm_params* p, const void* f_in_dev, void* f_tmp_dev, void* stream);
/* The push form of the same propagate (Sec. 4, "push" vs "pull"): every site moves its own
 * 37 populations to (x + vx_i mod lx, y + vy_i), dropping moves that leave the fluid.  Reads
 * are aligned and writes are shifted, the opposite of the pull form.  It writes exactly the
 * entries lbm_propagate writes, with the same values (a copy, so bit-identical), and
 * leaves the same entries for lbm_bc.  Same arguments, layout and errors as lbm_propagate. */
int32_t lbm_propagate_push(const lbm_params* p, const void* f_in_dev, void* f_tmp_dev, void* stream);
int32_t lbm_bc(const lbm_params* p, const void* f_in_dev, void* f_tmp_dev, void* stream);
int32_t lbm_collide(const lbm_params* p, const void* f_tmp_dev, void* f_out_dev, void* stream);

/* Macroscopic fields of a state (eq. "macro"): rho = sum f, rho u = sum xi f,
 * D rho T = sum |xi - u|^2 f.  Outputs are [lx][ly] doubles. */
int32_t lbm_moments(const lbm_params* p, const void* f_dev, double* rho_dev, double* ux_dev,
                    double* uy_dev, double* T_dev, void* stream);

/* Bytes of scratch lbm_kinetic_energy needs for this lattice. */
int64_t lbm_reduce_scratch_bytes(const lbm_params* p);

/* Total kinetic energy sum over fluid sites of rho |u|^2 / 2 (moments of eq. "macro"),
 * written to *out_dev.  Deterministic: per-block partial sums go to scratch_dev
 * (>= lbm_reduce_scratch_bytes bytes, device memory owned by the caller) and are then
 * summed in a fixed order by one block. */
int32_t lbm_kinetic_energy(const lbm_params* p, const void* f_dev, double* out_dev,
                           void* scratch_dev, size_t scratch_bytes, void* stream);

/* Kinetic energy exactly as lbm_kinetic_energy, for callers that cannot allocate device
 * memory while they run (for example an application whose device memory is all reserved
 * up front by its own pool, or a time-critical stepping loop that must not call cudaMalloc,
 * which can synchronise the device).  The paper has no counterpart: this is a library
 * convenience.  Nothing is allocated: the per-tile partial sums go to a fixed array of
 * LBM_NOALLOC_MAX_TILES doubles (2 MiB) built into the library, which every GPU that loads
 * the library holds until the process exits.  A lattice needs ceil(ly/32) * ceil(lx/4)
 * tiles (4096 x 8192 needs exactly the maximum); larger lattices return LBM_ESIZE.
 * The first call on each device looks up the array's device address (and may load the
 * library's device code); make that first call before any stream capture.  The address is
 * kept for the life of the process: after cudaDeviceReset on a device, do not call this
 * entry point on that device again (the array may have moved).  All calls share
 * the array and leave their partial sums in it; each call only reads what it has just
 * written, so no clearing is needed, but calls whose kernels can overlap on the GPU (on
 * different streams without ordering) race on it. */
#define LBM_NOALLOC_MAX_TILES 262144
int32_t lbm_kinetic_energy_noalloc(const lbm_params* p, const void* f_dev, double* out_dev, void* stream);

/* End-to-end run from host memory (synchronous): copies the four initial fields from
 * host (pinned for best speed) to fields_dev (4 * lx * ly doubles, device), builds the
 * equilibrium state in f_a_dev, runs n_steps fused steps between f_a_dev and f_b_dev,
 * computes the moments into fields_dev and copies them back to the four *_out_host
 * arrays.  Returns after the last copy has finished. */
int32_t lbm_simulate_host(const lbm_params* p, const double* rho_host, const double* ux_host,
                          const double* uy_host, const double* T_host, int32_t n_steps,
                          double* rho_out_host, double* ux_out_host, double* uy_out_host,
                          double* T_out_host, void* f_a_dev, void* f_b_dev, double* fields_dev,
                          void* stream);

/* ---- Layout comparison (Sec. 4: AoS, SoA, CSoA, CAoSoA), FP64 fused step, walls ----
 * LBM_LAYOUT_SOA is the layout of every other entry point: element (i, x, y) at
 * (i * lx + x) * pitch + y.  With pitch a multiple of 32 it is also the paper's CSoA
 * ("Cluster Structure of Array") with cluster width VL = 32 = the warp: every run of 32
 * consecutive y of one population is one aligned 256-byte cluster.
 * LBM_LAYOUT_AOS stores the 37 populations of a site contiguously: element (i, x, y) at
 * (x * pitch + y) * 37 + i.
 * The two partitioned layouts split each column into 32 partitions of P = pitch / 32 rows;
 * row y = k * P + j is element k of cluster j (the paper's CAoSoA partitioning):
 *   LBM_LAYOUT_PSOA   keeps one array per population: element (i, x, y) at
 *                     ((i * lx + x) * P + j) * 32 + k;
 *   LBM_LAYOUT_CAOSOA ("Clustered Array of Structure of Array") keeps the 37 clusters of
 *                     one (x, j) adjacent: element (i, x, y) at ((x * P + j) * 37 + i) * 32 + k.
 * Same buffer size (lbm_buffer_bytes) in every layout. */
enum lbm_layout { LBM_LAYOUT_SOA = 0, LBM_LAYOUT_AOS = 1, LBM_LAYOUT_PSOA = 2, LBM_LAYOUT_CAOSOA = 3 };
/* dst = src re-laid out between SoA and one of AOS, PSOA, CAOSOA (either direction); dst
 * and src must not be the same.  Exact copy. */
int32_t lbm_convert_layout(const lbm_params* p, int32_t from, const void* src_dev, int32_t to, void* dst_dev,
                           void* stream);
/* One fused step of a state stored in layout AOS, PSOA or CAOSOA (the same arithmetic as
 * lbm_step on the same gathered values; results agree with lbm_step up to the compiler's
 * contraction of multiply-adds). */
int32_t lbm_step_layout(const lbm_params* p, int32_t layout, const void* f_in_dev, void* f_out_dev, void* stream);

/* ---- Adjoint (reverse mode) of the FP64 step, for gradients of observables ----
 * The paper steps forward only; these are the transposed Jacobians of the same operations
 * (propagate and bc are linear, collide is differentiated site by site through the
 * moments of eq. "macro", the gravity shift and the Hermite equilibrium).  FP64 only. */
/* Bytes of workspace lbm_adjoint_step needs: 2 * lx * 26 doubles of wall slots (the
 * adjoint values fed from ghost rows, per wall and source column) plus per-tile partials. */
int64_t lbm_adjoint_work_bytes(const lbm_params* p);
/* lam_n = (d step / d f_n)^T lam_next, and *dtau_accum += lam_next . d step(f_n) / d tau
 * (deterministic per-tile partials summed in a fixed order).  f_n is the state the forward
 * step started from (recomputed or checkpointed by the caller); lam_* are state-shaped
 * buffers; work_dev holds lbm_adjoint_work_bytes bytes.  lam_n must not alias lam_next. */
int32_t lbm_adjoint_step(const lbm_params* p, const void* f_n_dev, const void* lam_next_dev, void* lam_n_dev,
                         double* dtau_accum_dev, void* work_dev, size_t work_bytes, void* stream);
/* lam = d E / d f for the total kinetic energy E = sum 1/2 rho |u|^2 of state f. */
int32_t lbm_kinetic_energy_grad(const lbm_params* p, const void* f_dev, void* lam_dev, void* stream);
/* Gradients of the initial fields of lbm_init against lam0 = dL/df^0:
 * g_X = sum_i lam0_i d f_i^eq(rho, u, T) / dX for X in (rho, ux, uy, T); [lx][ly] doubles. */
int32_t lbm_init_adjoint(const lbm_params* p, const double* rho_dev, const double* ux_dev, const double* uy_dev,
                         const double* T_dev, const void* lam0_dev, double* g_rho_dev, double* g_ux_dev,
                         double* g_uy_dev, double* g_T_dev, void* stream);

/* ---- Batched stepping of many independent lattices (uneven sizes, own tau, walls...) ----
 * The paper steps one lattice per process; this runs many independent problems in one
 * launch so that small lattices fill the GPU (its start-up mini-benchmark tuning, Sec. 6,
 * becomes the autotuner below).  All lattices of a batch share precision (LBM_FP64,
 * LBM_FP64_FIXED, LBM_FP32_SHIFTED or LBM_FP32_CONSERVED) and bc mode; each has its own lbm_params and its own
 * two state buffers.  Results are bit-identical to lbm_run on each lattice. */
typedef struct lbm_batch lbm_batch;
enum lbm_batch_mode {
  LBM_BATCH_PER_STEP = 1,   /* one launch per step over every strip of every lattice */
  LBM_BATCH_PERSISTENT = 2, /* one cooperative launch for all steps, grid barrier between steps */
  LBM_BATCH_LOOP = 3        /* the single-lattice kernel launched per lattice (baseline) */
};
/* Validates n lattices and binds their buffers (f_a_dev[j], f_b_dev[j]: device states of
 * lbm_buffer_bytes(&params[j]) bytes, current state in f_a; no two of the 2n buffers may
 * overlap, else LBM_EINVAL).  Allocates the batch's own
 * device descriptor table, tile table and barrier word (freed by lbm_batch_destroy).
 * Synchronous.  Default configuration: one launch per step, tiles of 32 x 4.  At most 65535
 * lattices. */
int32_t lbm_batch_plan(const lbm_params* params, void* const* f_a_dev, void* const* f_b_dev, int32_t n,
                       lbm_batch** out);
/* Sets mode, tile shape (a block steps a tile of 32 rows x tile_columns columns, one warp
 * per column; tile_columns = 1, 2, 4 or 8) and blocks per SM (persistent only; 0 = all that
 * fit).  Synchronous when the tile shape changes (the tile table is rebuilt). */
int32_t lbm_batch_configure(lbm_batch* b, int32_t mode, int32_t tile_columns, int32_t blocks_per_sm);
/* Reads the configuration (blocks_per_sm: the value the persistent launch uses, else 0). */
int32_t lbm_batch_config(const lbm_batch* b, int32_t* mode, int32_t* tile_columns, int32_t* blocks_per_sm);
/* Times every candidate configuration for trial_steps steps (after one warm-up step each)
 * and keeps the fastest.  Candidates: per-step launches with tiles of 2, 4 and 8 columns;
 * for batches of at most 2^20 sites also the persistent launch with those tiles and the
 * two largest block counts per SM (on larger batches its L1-bypassing loads cost more
 * than the kernel boundaries it saves).  It ADVANCES the batch by (trial_steps + 1) steps per candidate:
 * call it before initialising the states, or on states whose evolution does not matter.
 * Synchronous. */
int32_t lbm_batch_autotune(lbm_batch* b, int32_t trial_steps, void* stream);
/* n_steps steps of every lattice in the current configuration; stream-ordered. */
int32_t lbm_batch_run(lbm_batch* b, int32_t n_steps, void* stream);
/* Which buffer holds the current states: 0 = f_a, 1 = f_b (flips with every odd run). */
int32_t lbm_batch_parity(const lbm_batch* b);
/* Total fluid sites of the batch. */
int64_t lbm_batch_sites(const lbm_batch* b);
/* Synchronous: LBM_OK, or LBM_ETIMEOUT if the grid-barrier wait of any persistent run since
 * the previous call expired (that run stopped early and the states are undefined); clears
 * the flag.  A later run does not erase an earlier run's timeout. */
int32_t lbm_batch_status(lbm_batch* b);
/* Grid-barrier wait limit in ns (default 2 s, at most 60 s).  phantom_arrivals makes every
 * barrier wait for that many extra blocks that never arrive: a test hook that forces the
 * wait to expire (0 in normal use). */
int32_t lbm_batch_set_wait(lbm_batch* b, int64_t timeout_ns, int32_t phantom_arrivals);
void lbm_batch_destroy(lbm_batch* b);

/* ---- Peak probes: the roofline denominators of the arithmetic pipes, measured ----
 * Runs a probe kernel on the current device (8 blocks of 256 threads per SM, each thread
 * 8 independent dependency chains of 4096 operations) and returns the sustained rate in
 * *ops_per_second (operations, not flops: one FMA is one operation).  kind: 0 = float64
 * FMA, 1 = float32 FMA, 2 = 32-bit integer multiply-add, 3 = signed 64 x 64 -> high 64
 * product (__mul64hi), 4 = unsigned one.  Synchronous (device-wide); allocates and frees a
 * small result buffer; returns LBM_EINVAL for another kind. */
enum lbm_probe { LBM_PROBE_DFMA = 0, LBM_PROBE_FFMA = 1, LBM_PROBE_IMAD = 2, LBM_PROBE_MULHI64 = 3,
                 LBM_PROBE_UMULHI64 = 4 };
int32_t lbm_probe_peak(int32_t kind, double* ops_per_second);

/* Human-readable text of an lbm_status code. */
const char* lbm_strerror(int32_t status);
/* The CUDA error code behind the most recent LBM_ECUDA on this thread (0 if none). */
int32_t lbm_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_D2Q37_H */
