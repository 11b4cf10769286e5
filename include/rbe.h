/*
 * rbe.h -- C ABI of librbe, a GB300 (sm_103a) implementation of the per-step
 * force evaluation of the random batch Ewald (RBE) method of Jin, Li, Xu and
 * Zhao, "A random batch Ewald method for particle systems with Coulomb
 * interactions" (arXiv:2010.01559).
 *
 * What one force evaluation computes (paper section / equation):
 *   - P wave vectors k = 2 pi m / L, m in Z^3 \ {0}, drawn i.i.d. from the
 *     discrete Gaussian P_k = exp(-k^2 / 4 alpha) / S            (Eq. probexpression)
 *     with S = H^3 - 1                                          (Eq. S, Eq. psf);
 *   - the structure factors rho(k_l) = sum_j q_j exp(i k_l . r_j)        (Sec. 2);
 *   - the RBE Fourier force
 *       F*_i = -sum_l (S/P) 4 pi q_i k_l / (V k_l^2) Im(e^{-i k_l.r_i} rho(k_l))
 *                                                                (Eq. rbmapprox);
 *   - the real-space force -q_i sum_j q_j G(r) r_ij / r under the cutoff r_c,
 *     G(r) = erfc(sqrt(alpha) r)/r^2 + 2 sqrt(alpha) exp(-alpha r^2)/(sqrt(pi) r)
 *                                                           (Eq. force, 2nd term);
 *   - a shifted Lennard-Jones force                           (Eq. Ljpotential);
 *   - optionally the energy (FP64): frozen-batch estimator of U_1 (Sec. 2 with
 *     the S/P weights of Eq. rbmapprox), self term -sqrt(alpha/pi) sum q^2,
 *     neutralising background -pi (sum q)^2 / (2 V alpha), truncated U_2, LJ;
 *   - optionally dE/dq_i (the electrostatic potential at particle i).
 * One MD step (rbe_step) adds the Langevin thermostat of Sec. 3.3 as a kick /
 * exact Ornstein-Uhlenbeck / drift update, closing the loop of Algorithm 1
 * (or the Andersen / Nose-Hoover variants); its real-space pairs come from a
 * Verlet neighbour list kept on the device (rbe_step_ex).
 *
 * Conventions for every entry point:
 *   - Array pointers are caller-owned DEVICE memory (except the *_host entry
 *     points), 16-byte aligned, contiguous.  The library owns only its
 *     workspace, allocated by rbe_create / rbe_create_batch for n_max
 *     particles and freed by rbe_destroy.
 *   - Particles are float4 / double4 records (x, y, z, q); positions may lie
 *     anywhere, they are wrapped into the periodic cube [0, L)^3 internally.
 *     Forces are float4 / double4 records (Fx, Fy, Fz, 0).
 *   - Work is enqueued on the handle's CUDA stream (rbe_set_stream; default:
 *     the legacy default stream) and the calls return without synchronising,
 *     except the *_host entry points and rbe_sync.
 *   - No exception crosses the ABI; every call returns an rbe_status.  Argument
 *     errors are detected on the host before anything is enqueued.  CUDA errors
 *     are reported as RBE_ERR_CUDA.  Device-side conditions (a k-sample that
 *     exhausted its 32 attempts, an overflowing neighbour list, a NaN or
 *     infinite input) are latched in a device word and reported by the next
 *     rbe_sync (or *_host call).  rbe_last_error(h) gives a message.
 *   - Units are the caller's; coulomb_prefactor multiplies every Coulomb term
 *     (1 in the reduced units of Sec. 4.1, the Bjerrum length in Sec. 4.2).
 */
#ifndef RBE_H
#define RBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rbe_ctx *rbe_handle;

typedef enum {
    RBE_OK = 0,
    RBE_ERR_ARG = 1,        /* invalid argument (null pointer, size, parameter range) */
    RBE_ERR_CUDA = 2,       /* a CUDA runtime call failed                              */
    RBE_ERR_OOM = 3,        /* device allocation failed                                */
    RBE_ERR_SAMPLER = 4,    /* a k-sample hit (0,0,0) on 32 attempts in a row           */
    RBE_ERR_TIMEOUT = 5,    /* a host wait ran past the handle's wait limit
                               (rbe_set_wait_limit); the work is still queued          */
    RBE_ERR_NONFINITE = 6,  /* a position or charge of an input was NaN or infinite
                               (latched on the device, reported at the next sync)     */
    RBE_ERR_STATE = 7,      /* call not valid for this handle (e.g. wrong n for a batch) */
    RBE_ERR_LIST = 8,       /* a particle had more neighbours within r_c + skin than the
                               list holds (a much denser region than the mean density):
                               the steps since the last rbe_sync missed pairs; run with
                               skin < 0 (no list) or a smaller skin */
    RBE_ERR_BOUNDS = 9      /* only in the bounds-checked build (RBE_CHECK_BOUNDS): an
                               index computed on the device fell outside its array; the
                               access was skipped and the results are not meaningful */
} rbe_status;

enum { RBE_FP64 = 0, RBE_MIXED = 1 };

/* k-samplers (rbe_params.sampler).  RBE_SAMPLER_EXACT: P i.i.d. samples per
 * step by an integer inverse-CDF table per axis, a pure function of (seed,
 * stream, step, l).  RBE_SAMPLER_MH: the paper's Metropolis-Hastings sampler
 * (Sec. 3.1): three per-axis independence chains with the rounded-Gaussian
 * proposal, (0,0,0) triples discarded, consumed in order across evaluations
 * (the set K of Algorithm 1); the chain state lives in the handle and starts
 * at m = 0, iteration 0. */
enum { RBE_SAMPLER_EXACT = 0, RBE_SAMPLER_MH = 1 };

/* Thermostats of rbe_step (rbe_params.thermostat).  RBE_THERMO_LANGEVIN:
 * kick, exact Ornstein-Uhlenbeck with friction gamma, drift (Sec. 3.3).
 * RBE_THERMO_ANDERSEN: the loop step of Algorithm 1 as printed -- leapfrog
 * (kick, drift) and then, with probability andersen_nu * dt per particle, a
 * new velocity drawn from N(0, kT/m).
 * RBE_THERMO_NOSE_HOOVER: the deterministic thermostat whose equations of
 * motion Sec. 3.3 states (dr/dt = v, m dv/dt = F - xi m v, dxi/dt =
 * (sum m |v|^2 - 3 N kT) / Q) and leaves for later work; Q = 3 N kT nh_tau^2.
 * Discretised as a leapfrog: xi advances from the previous step's sum m|v|^2
 * (not on the first step after creation or rbe_nose_hoover_xi(..., set=1)),
 * then v <- [v (1 - xi dt/2) + (dt/m) F] / (1 + xi dt/2) and the drift.  The
 * kinetic sum is accumulated in 64-bit fixed point (m|v|^2 / kT in units of
 * 2^-32), so runs are deterministic. */
enum { RBE_THERMO_LANGEVIN = 0, RBE_THERMO_ANDERSEN = 1, RBE_THERMO_NOSE_HOOVER = 2 };

/* Parts selectable in rbe_forces_ex. */
enum { RBE_PART_FOURIER = 1, RBE_PART_REAL = 2, RBE_PART_LJ = 4, RBE_PART_ALL = 7 };

/* Parameters of one periodic system (cubic box, reduced units).  144 bytes. */
typedef struct {
    double box;               /* L > 0: edge of the cubic periodic box (Sec. 2)          */
    double alpha;             /* Ewald splitting parameter, erfc(sqrt(alpha) r) (Sec. 2) */
    double r_c;               /* real-space cutoff, 0 < r_c <= L/2 (minimum image); cells of
                                 side >= r_c + skin, or one cell (all pairs) when
                                 r_c + skin > L/3                                         */
    double coulomb_prefactor; /* multiplies all Coulomb terms (Sec. 4.1: 1)              */
    double lj_eps;            /* shifted-LJ epsilon; 0 disables LJ (Eq. Ljpotential)     */
    double lj_sigma;          /* LJ sigma (r_off = 0)                                    */
    double lj_rcut;           /* LJ cutoff R_c (<= r_c); V_shift makes V(R_c) = 0         */
    double gamma;             /* Langevin friction (Sec. 3.3)                            */
    double kT;                /* temperature 1/beta (k_B = 1)                            */
    double dt;                /* time step                                               */
    double mass;              /* particle mass (all particles)                           */
    uint64_t seed;            /* Philox key of this system                               */
    uint32_t stream;          /* Philox stream id (distinct per replica)                 */
    int32_t P;                /* batch size p >= 1 (Eq. rbmapprox)                        */
    int32_t n_max;            /* capacity in particles (single-system handles)           */
    int32_t precision;        /* RBE_MIXED (default path of rbe_step) or RBE_FP64         */
    double andersen_nu;       /* Andersen collision frequency nu, 0 <= nu dt <= 1          */
    int32_t sampler;          /* RBE_SAMPLER_EXACT (0) or RBE_SAMPLER_MH; one per handle  */
    int32_t thermostat;       /* RBE_THERMO_LANGEVIN (0), _ANDERSEN or _NOSE_HOOVER       */
    double nh_tau;            /* Nose-Hoover time constant, Q = 3 N kT nh_tau^2 (> 0 there) */
    double skin;              /* Verlet skin of rbe_step's neighbour list: 0 = automatic
                                 (0.1 r_c), < 0 = no list (every step scans the cells);
                                 at most L/3 - r_c (L/2 - r_c in the one-cell mode).  The
                                 cells of every path of the handle then have side
                                 >= r_c + skin                                          */
} rbe_params;

/* Derived constants of system `sys` of a handle (for inspection and tests). */
typedef struct {
    double H;                 /* sum_m exp(-pi^2 m^2 / (alpha L^2)) over |m| <= M (Eq. psf) */
    double S;                 /* H^3 - 1 (Eq. S)                                           */
    int32_t M;                /* per-axis table half-width: tail weight < 2^-64            */
    int32_t n_cells_dim;      /* cells per box edge of the real-space cell list            */
    int32_t n;                /* particles of this system (batch) or n_max (single)        */
    int32_t P;                /* batch size                                                */
    int32_t n_systems;        /* systems in the handle                                     */
    int32_t first_particle;   /* offset of this system in concatenated particle arrays     */
    int32_t first_k;          /* offset of this system in concatenated k arrays            */
    int32_t reserved;
} rbe_info;

/* Create a handle for one system of up to p->n_max particles.  Builds the
 * per-axis sampling table (Eq. probexpression, per-axis marginal) and S
 * (Eq. S) in FP64 on the host and allocates the device workspace.
 * Errors: RBE_ERR_ARG for out-of-range parameters (L, alpha, r_c, P <= 0,
 * r_c > L/2, lj_rcut > r_c, n_max < 0), RBE_ERR_OOM, RBE_ERR_CUDA. */
rbe_status rbe_create(const rbe_params *p, rbe_handle *out);

/* Create a handle for n_replicas independent systems (replica r has
 * per_replica[r] and n_per_replica[r] particles) evaluated together: every
 * kernel launch covers all replicas.  Particle arrays passed to the batched
 * calls are the replicas' arrays concatenated in replica order; energies are
 * n_replicas x 4 doubles.  Same errors as rbe_create. */
rbe_status rbe_create_batch(const rbe_params *per_replica, const int32_t *n_per_replica,
                            int32_t n_replicas, rbe_handle *out);

/* Free the workspace and the handle (NULL is ignored).  Synchronises the stream. */
void rbe_destroy(rbe_handle h);

/* Message describing the last failure on h (thread-local global if h is NULL). */
const char *rbe_last_error(rbe_handle h);

/* Set the CUDA stream (a cudaStream_t) used for all work of h. */
rbe_status rbe_set_stream(rbe_handle h, void *cuda_stream);

/* Fill *info for system `sys` of h.  RBE_ERR_ARG for a bad index. */
rbe_status rbe_get_info(rbe_handle h, int32_t sys, rbe_info *info);

/* Copy system sys's per-axis sampling table (2M+1 uint64, host memory) to
 * table_out: entry j = floor(2^32 CDF(j - M)), last entry 2^32. */
rbe_status rbe_get_table(rbe_handle h, int32_t sys, uint64_t *table_out);

/* Draw the k-batch of step `step` for every system (Eq. probexpression):
 * m_out (device, int32, total-P x 4) receives (m_x, m_y, m_z, attempts) per
 * sample.  Sample l of a system uses Philox4x32-10 with key (seed_lo, seed_hi)
 * and counter (l, attempt, step_lo, (stream << 8) | 1); each 32-bit word maps
 * to one axis by the integer table; (0,0,0) is discarded and redrawn
 * (Sec. 3.1), at most 32 attempts.  With RBE_SAMPLER_MH the batch depends on
 * the chains' history, not on `step`: m_out receives the batch of the last
 * evaluation (attempts field 1), and the chains do not advance. */
rbe_status rbe_sample_k(rbe_handle h, uint64_t step, int32_t *m_out);

/* One RBE force evaluation, mixed precision (FP32 phases / sincos / forces
 * from exact 32-bit fixed-point fractional coordinates; FP64 rho(k) sums and
 * energies).  n: number of particles (== n_max-capacity-bounded; for a batch
 * handle, the total).  pos_q: float4[n].  step selects the k-batch.
 * F_out: float4[n] total force.  E_out (nullable): double[4 * n_systems] =
 * {total, Fourier incl. self and background, real-space Coulomb, LJ}.
 * phi_out (nullable): float[n], dE/dq_i. */
rbe_status rbe_forces(rbe_handle h, int32_t n, const float *pos_q, uint64_t step,
                      float *F_out, double *E_out, float *phi_out);

/* As rbe_forces, restricted to the parts in `parts` (RBE_PART_* mask);
 * energies and phi of the parts left out are zero. */
rbe_status rbe_forces_ex(rbe_handle h, int32_t n, const float *pos_q, uint64_t step,
                         int32_t parts, float *F_out, double *E_out, float *phi_out);

/* The plain FP64 path: the same steps with FP64 positions, phases, sincos,
 * erfc and sums throughout.  pos_q: double4[n], F_out: double4[n],
 * phi_out: double[n]. */
rbe_status rbe_forces_f64(rbe_handle h, int32_t n, const double *pos_q, uint64_t step,
                          int32_t parts, double *F_out, double *E_out, double *phi_out);

/* nsteps MD steps (Algorithm 1 with the Langevin thermostat of Sec. 3.3),
 * mixed precision, updating pos_q (float4[n]) and vel (float4[n], w unused)
 * in place.  step_dev (device uint64) holds the index of the next step; each
 * step reads it to select its k-batch and noise and increments it on the
 * device, so a captured replay advances the stream.  The step sequence is
 * replayed from a CUDA graph when use_graph was enabled (rbe_set_graph). */
rbe_status rbe_step(rbe_handle h, int32_t n, float *pos_q, float *vel, int32_t nsteps,
                    uint64_t *step_dev);

/* rbe_step that also writes each step's total force (float4[n], caller order,
 * w = 0) to F_out (nullable); after the call F_out holds the last step's
 * force, evaluated at the positions that step started from.
 *
 * Neighbour list (mixed steps, skin >= 0): the real-space pairs of a step come
 * from a list of the pairs within r_c + skin built on the device whenever some
 * particle has moved more than skin/2 (minimum image) since the last build --
 * then every pair within r_c is still in the list, so the step's forces equal
 * those of a full cell scan up to FP32 summation order.  Each step's first
 * kernel tests the displacements of the positions it is given, so positions
 * changed by the caller between calls are also caught; any other evaluation
 * on the handle (forces, FP64 steps, observables, autotune) forces a rebuild
 * at the next step.  A list overflow is latched and reported by rbe_sync as
 * RBE_ERR_LIST. */
rbe_status rbe_step_ex(rbe_handle h, int32_t n, float *pos_q, float *vel, int32_t nsteps,
                       uint64_t *step_dev, float *F_out);

/* Neighbour-list statistics since the handle was created (synchronises h's
 * stream): builds, the number of list builds; max_count, the largest number of
 * neighbours within r_c + skin any particle had at a build; capacity, the
 * entries each particle's list holds (0 when the handle has no list). */
rbe_status rbe_list_stats(rbe_handle h, int64_t *builds, int32_t *max_count, int32_t *capacity);

/* FP64 MD steps: pos_q, vel double4[n]. */
rbe_status rbe_step_f64(rbe_handle h, int32_t n, double *pos_q, double *vel, int32_t nsteps,
                        uint64_t *step_dev);

/* Nose-Hoover friction xi of every system (double[n_systems], host).
 * set = 0: read the current values into xi (synchronises h's stream).
 * set = 1: replace them with xi (e.g. to resume a run); the next step then
 * uses them as given and advances them from its own kinetic sum afterwards.
 * Systems with another thermostat carry a xi that no step uses.  Errors:
 * RBE_ERR_ARG (null handle or xi), RBE_ERR_CUDA. */
rbe_status rbe_nose_hoover_xi(rbe_handle h, double *xi, int32_t set);

/* Enable (1) or disable (0) CUDA-graph replay of rbe_step.  The first
 * rbe_step call after enabling captures one step per distinct argument set. */
rbe_status rbe_set_graph(rbe_handle h, int32_t use_graph);

/* Host-memory variants: copy the inputs from host (preferably pinned)
 * memory, run, copy the outputs back and synchronise.  Staging buffers are
 * the handle's own.  rbe_forces_host: pos_q float4[n] in, F_out float4[n]
 * out, E_out (nullable) double[4 n_systems] out.  rbe_step_host: pos_q and
 * vel float4[n] in/out, steps step0 .. step0 + nsteps - 1; when both arrays
 * are page-locked (cudaHostAlloc, cudaHostRegister) the step's kernels read
 * and write them in place over the host link instead of staging copies, and
 * on a neighbour-list handle the call returns as soon as the step's closing
 * kernel has written a completion word to the handle's mapped host memory
 * (every output store is visible to the host by then; the kernel's last
 * blocks may still be retiring, and later work on h's stream is ordered
 * after them as usual).  Errors as rbe_step and rbe_sync. */
rbe_status rbe_forces_host(rbe_handle h, int32_t n, const float *pos_q, uint64_t step,
                           float *F_out, double *E_out);
rbe_status rbe_step_host(rbe_handle h, int32_t n, float *pos_q, float *vel, int32_t nsteps,
                         uint64_t step0);

/* Synchronise h's stream and report latched device conditions
 * (RBE_ERR_SAMPLER, RBE_ERR_LIST, RBE_ERR_NONFINITE, RBE_ERR_BOUNDS) and
 * asynchronous CUDA errors.  Clears the latch. */
rbe_status rbe_sync(rbe_handle h);

/* Failure detection on the host side: the longest time, in seconds, that a
 * call of h waiting for the GPU (rbe_sync, rbe_forces_host, rbe_step_host)
 * may wait (0, the default: no limit).  When it passes, the call returns
 * RBE_ERR_TIMEOUT at once; the work stays queued on h's stream and the
 * caller must call rbe_sync (which waits again, under the same limit) before
 * reading or freeing the buffers of the call.  Not an RBE operation: it lets
 * an MD driver notice a GPU that stopped answering without blocking forever.
 * Errors: RBE_ERR_ARG for a null handle or a negative or non-finite limit. */
rbe_status rbe_set_wait_limit(rbe_handle h, double seconds);

/* Launch shapes of the per-particle kernels (0 = automatic for every field). */
typedef struct {
    int32_t rho_chunk;     /* particles per structure-factor chunk: power of two in [32, 8192] */
    int32_t force_split;   /* threads per particle in the Fourier-force pass: 1, 2, 4 or 8     */
    int32_t real_split;    /* threads per particle in the mixed real-space pass: 1, 3 or 9,
                              each scanning 9 / real_split of the 9 neighbour rows (the FP64
                              pass uses the largest power of two not above it)             */
    int32_t real_seg;      /* cells along x per real-space block: 1 .. cells per edge           */
    int32_t list_split;    /* threads per particle in the neighbour-list pass of rbe_step:
                              1, 2, 4 or 8                                                   */
} rbe_tuning;

/* Set the launch shapes (results change only by floating-point summation
 * order).  RBE_ERR_ARG for a value out of range. */
rbe_status rbe_set_tuning(rbe_handle h, const rbe_tuning *t);

/* The launch shapes in effect for the last prepared particle count (automatic
 * choices resolved). */
rbe_status rbe_get_tuning(rbe_handle h, rbe_tuning *t);

/* Fusion of a mixed-precision list MD step (rbe_step*, rbe_step_ex): with
 * on = 1 the structure factors (Eq. rbmapprox's rho(k)) and the real-space
 * pass over a standing neighbour list run as one launch whose blocks take
 * either kind of work, so that every SM runs both; with on = 0 they are two
 * launches on two streams; with on = -1 (the default) rbe_autotune times a
 * list evaluation both ways and keeps the faster, and before any autotune
 * systems of 2^19 particles and more (over all replicas) fuse.  The results
 * are the same to the last bit either way.  Captured step graphs are
 * dropped.  RBE_ERR_ARG unless on is -1, 0 or 1. */
rbe_status rbe_set_fusion(rbe_handle h, int32_t on);

/* *on = 1 if a list MD step at the current particle count runs fused, else 0. */
rbe_status rbe_get_fusion(rbe_handle h, int32_t *on);

/* Time the candidate launch shapes of each tunable kernel on the given input
 * (device pos_q, n particles) with CUDA events, keep the fastest and return
 * them in *out (nullable).  With a neighbour list and fusion automatic it also
 * chooses between the fused and the separate list step (rbe_set_fusion). */
rbe_status rbe_autotune(rbe_handle h, int32_t n, const float *pos_q, rbe_tuning *out);

/* Kernels of one evaluation, in launch order (per-kernel profile indices). */
enum {
    RBE_K_PREP = 0,          /* fixed-point coordinates, cell ids, charge sums      */
    RBE_K_SCAN = 1,          /* exclusive scan of cell counts, step latch           */
    RBE_K_SCATTER = 2,       /* counting-sort scatter                               */
    RBE_K_CELL_ORDER = 3,    /* order inside each cell by original index            */
    RBE_K_RHO = 4,           /* k-sampling, per-chunk structure factors, and (last
                                block of each k-tile) FP64 rho(k), energy terms,
                                force coefficients                                */
    RBE_K_FINALIZE = 5,      /* reserved (finalisation is fused into RBE_K_RHO)     */
    RBE_K_FOURIER_FORCE = 6, /* RBE Fourier force and dE/dq (Eq. rbmapprox)         */
    RBE_K_REAL = 7,          /* real space + LJ + assembly (+ Langevin)             */
    RBE_K_ENERGY = 8,        /* FP64 energy reduction                               */
    RBE_K_LIST_BUILD = 9,    /* neighbour-list build (list MD steps; returns at once
                                when no particle moved beyond skin/2)             */
    RBE_K_RHO_LIST = 10,     /* list MD steps with fusion on: RBE_K_RHO and the pass
                                over a standing neighbour list in one launch       */
    RBE_K_COUNT = 11
};

/* Enable (1) or disable (0) per-kernel timing.  While enabled, rbe_forces*,
 * rbe_step* run every kernel of an evaluation on the handle's stream, one
 * after another (the concurrent branches are serialised, so each time is the
 * kernel's alone), record CUDA events around each, wait for them at the end of
 * each evaluation and accumulate the device time per kernel; graph replay is
 * bypassed. */
rbe_status rbe_profile(rbe_handle h, int32_t enable);

/* Read and reset the accumulated profile: ms[RBE_K_COUNT] device milliseconds
 * and launches[RBE_K_COUNT] (either may be NULL). */
rbe_status rbe_profile_read(rbe_handle h, double *ms, int64_t *launches);

/* Kernels launched through h since it was created (graph replays count the
 * kernels of the replayed step). */
rbe_status rbe_launch_count(rbe_handle h, int64_t *count);

/* True (non-random) energy and pressure of a configuration, the observables
 * the paper evaluates "without random batch": the full Ewald sum over the
 * cube 0 < |m|_inf <= mmax (mmax <= 0: the sampler's M, tail below 2^-64),
 * the real-space and LJ parts under their cutoffs, the kinetic energy of
 * `vel`, and the virial W = -dE/dlambda under r -> lambda r, L -> lambda L:
 *   real space  sum_{i<j} lB q_i q_j [erfc(sqrt(a) r)/r + 2 sqrt(a/pi) e^{-a r^2}]
 *   Fourier     sum_k A_k |rho_k|^2 (1 - k^2/(2 alpha)),
 *               A_k = (2 pi lB / V) e^{-k^2/(4 alpha)} / k^2
 *   background  3 E_bg;   LJ  sum_{i<j} r.F_ij
 * P = (2 E_kin + W) / (3 V).  Structure factors use the mixed path's phases
 * (FP32 sin/cos of exact 32-bit phases), sums in FP64.
 * pos_q: device float4[n] (x, y, z, q); vel: device float4[n] or NULL (E_kin
 * = 0).  out: HOST double[12 * systems], per system: E_total, E_fourier (incl.
 * self and background), E_real, E_lj, E_kin, W_fourier, W_real, W_lj,
 * W_background, pressure, kinetic temperature 2 E_kin / (3 n), 0.  Synchronous.
 * Errors: RBE_ERR_ARG (NULL, n, mmax above 2^24 wave vectors), RBE_ERR_OOM,
 * RBE_ERR_CUDA. */
rbe_status rbe_observables(rbe_handle h, int32_t n, const float *pos_q, const float *vel,
                           int32_t mmax, double *out);

/* Measured throughput of the two units the hot path leans on, for rooflines:
 * the special-function unit (sin/cos results, as the Fourier passes use them)
 * and the FP32 FMA pipe, per SM per clock, from short saturating probe kernels
 * on the current device (about 10 ms; allocates and frees 1 MB).  sm_clock_mhz
 * is the clock over the probe (SM cycles counted in the probe / its duration).
 * Not an RBE operation: it turns counters into fractions of what this GPU can
 * do.  Errors: RBE_ERR_ARG for a NULL out, RBE_ERR_CUDA. */
typedef struct {
    double sfu_per_clk_sm;    /* __sincosf results (sin and cos each count 1) per SM per clock */
    double ffma_per_clk_sm;   /* FP32 FMA instructions per SM per clock                      */
    double sm_clock_mhz;      /* SM clock measured during the probe                         */
    int32_t sms;              /* streaming multiprocessors                                  */
} rbe_peaks;
rbe_status rbe_probe_peaks(rbe_peaks *out);

/* Fourier part of one RBE evaluation without any device allocation, for
 * callers that cannot call cudaMalloc: an MD engine whose memory pool owns all
 * device memory and forbids plugins to allocate, or a latency-bound loop that
 * cannot afford cudaMalloc's implicit device-wide synchronisation.  The paper has no counterpart: this is an
 * interface variant of rbe_forces_ex(..., RBE_PART_FOURIER, ...) that needs no
 * handle.
 *
 * p: system parameters (box, alpha, P, seed, stream, coulomb_prefactor are
 * used; sampler must be RBE_SAMPLER_EXACT, the i.i.d. draws of Sec. 3.1, else
 * RBE_ERR_ARG).  pos_q: device float4[n] (x, y, z, q), caller-owned.  F_out:
 * device float4[n] receives the RBE Fourier force (caller's order).  E_out
 * (device, nullable): one double, the Fourier energy including self and
 * background terms.  n = 0 without E_out returns RBE_OK at once (nothing to
 * compute).  cuda_stream: a cudaStream_t or NULL.  The k-batch of `step` is
 * the same one rbe_forces draws for the same parameters.
 *
 * Scratch: a 4 MiB file-scope device array inside librbe, held by every GPU
 * that loads the library until the process exits.  Limits, checked on the host
 * (RBE_ERR_ARG with a message from rbe_last_error(NULL)): finite box, alpha
 * and coulomb_prefactor, 1 <= P <= 1024, a
 * sampling table of at most 4096 entries, and n * P small enough that the
 * per-chunk partial sums fit (chunks of up to 65536 particles; e.g. n = 2^20
 * with P = 500 fits).  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  Every call shares the array and
 * overwrites what it reads, so no state carries over between calls, but calls
 * that overlap on the GPU (e.g. on two streams) race on it and must be
 * serialised.  The call synchronises cuda_stream (not the device) before
 * returning; the error word (RBE_ERR_SAMPLER, RBE_ERR_NONFINITE for a NaN or
 * infinite input) is read back on that stream.  It calls
 * no cudaMalloc, cudaFree or other allocating routine. */
rbe_status rbe_fourier_forces_noalloc(const rbe_params *p, int32_t n, const float *pos_q,
                                      uint64_t step, float *F_out, double *E_out,
                                      void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* RBE_H */
