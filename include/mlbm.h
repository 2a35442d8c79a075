/*
 * mlbm.h — C ABI of the GB300 multi-level lattice Boltzmann library.
 *
 * The library advances the multi-level (grid-refined, ratio 2) lattice
 * Boltzmann method of Astoul, Wissocq, Boussuge, Sengissen & Sagaut,
 * "Analysis and reduction of spurious noise generated at grid refinement
 * interfaces with the lattice Boltzmann method" (arXiv 2004.11863):
 *   - per level, the fused stream-and-collide update of eq. LBMequation with
 *     the BGK collision (eq. BGKmodel), the projected regularized collision
 *     (eqs. reguProcedure, a1Proj, LBMscheme_reg) or the recursive
 *     regularized collision (eqs. f1RR, a13RR), on D2Q9 (Sec. 3.1), D3Q19 or
 *     D3Q27, with the third-order equilibrium of eq. fEqH;
 *   - between levels, the cell-vertex transfer of Sec. 4.3: coarse-to-fine
 *     temporal (eq. TempInt) and spatial (eq. spaceInt) interpolation with
 *     the rescaling of eq. rescff, and fine-to-coarse filtering
 *     (eq. filterFneq) with the rescaling of eq. rescfc; tau_f = 2 tau_c - 1/2
 *     (eq. rescTau).
 *
 * Every step runs in hand-written CUDA kernels for sm_103a.  Populations are
 * stored per level as structure-of-arrays planes of g_i = f_i - f0_i(rho0, U)
 * (FP32 or FP16; U = 0 is the rest-state shift f_i - w_i rho0), streamed in
 * place with the AA pattern.
 *
 * General rules
 *   - Every function returns 0 on success or a negative LBM_E* code; no
 *     function throws or aborts.  lbm_strerror() names a code.
 *   - A handle is used by one host thread at a time.  Work is issued on the
 *     CUDA stream given to lbm_create (0 = the legacy default stream) and is
 *     asynchronous unless a function says it synchronises.
 *   - The handle owns all device memory it allocates (through the optional
 *     allocator, else cudaMalloc) and frees it in lbm_destroy.  The caller
 *     owns every host buffer it passes; host buffers are only read or written
 *     during the call.
 *   - Level l has node counts n[3] (lbm_level_info).  Level arrays are
 *     ordered x fastest, then y, then z: index = (z*n[1] + y)*n[0] + x.
 *     Level 0 is periodic on every axis.  Level l >= 1 occupies the closed
 *     box box[l-1] given in level l-1 node units; an axis of the box that
 *     spans the whole periodic parent axis (lo = 0, hi = parent count) is
 *     periodic on level l with twice the parent's nodes, any other axis holds
 *     2 (hi - lo) + 1 nodes.  Macroscopic values are in each level's own
 *     lattice units (velocities are equal across levels, Sec. 4.1).
 */
#ifndef MLBM_H
#define MLBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define LBM_OK 0
#define LBM_EINVAL (-1)    /* invalid argument or layout */
#define LBM_ENOMEM (-2)    /* device or host allocation failed */
#define LBM_ECUDA (-3)     /* a CUDA runtime call or launch failed */
#define LBM_EUNSTABLE (-4) /* non-finite mass found by lbm_diag */
#define LBM_ESTATE (-5)    /* call out of order (e.g. step before init) */
#define LBM_ETIMEOUT (-6)  /* a bounded device-side wait ran out (lbm_set_fused) */

/* Lattices (Sec. 3.1; 3D sets of the same Hermite construction). */
#define LBM_D2Q9 0
#define LBM_D3Q19 1
#define LBM_D3Q27 2
/* Collisions: eq. BGKmodel; eqs. reguProcedure..LBMscheme_reg (REG);
 * eqs. f1RR, a13RR (RR); hybrid recursive regularized (H-RR, eq. a1ij_HRR:
 * a1 = sigma a1^(2) + (1 - sigma)(-2 tau rho cs^2 S), S from second-order
 * central differences of the pre-collision velocity, with the strain-rate
 * transfers of Sec. 4.4 at refinement interfaces). */
#define LBM_BGK 0
#define LBM_REG 1
#define LBM_RR 2
#define LBM_HRR 3
/* Population storage: g = f - w rho0 in binary32 or binary16 (compute is
 * always binary32). */
#define LBM_FP32_SHIFTED 0
#define LBM_FP16_SHIFTED 1

#define LBM_MAX_LEVELS 4

typedef struct lbm_ctx* lbm_handle;

/* Closed box [lo, hi] of a refined level, in parent-level node units. */
typedef struct {
  int lo[3];
  int hi[3];
} lbm_box;

typedef struct {
  int lattice;   /* LBM_D2Q9 | LBM_D3Q19 | LBM_D3Q27 */
  int collision; /* LBM_BGK | LBM_REG | LBM_RR | LBM_HRR */
  int storage;   /* LBM_FP32_SHIFTED | LBM_FP16_SHIFTED */
  double tau0;   /* level-0 relaxation time, > 1/2; level l uses
                    tau_l = 2 tau_{l-1} - 1/2 (eq. rescTau) */
  double rho0;   /* reference density of the shifted storage (usually 1) */
  int dims[3];   /* level-0 node counts; dims[2] = 1 for D2Q9 */
  int nlevels;   /* 1 .. LBM_MAX_LEVELS */
  lbm_box box[LBM_MAX_LEVELS - 1];
  int batch;     /* independent runs sharing this layout (>= 1); each run
                    has its own populations and initial state */
  double u_ref[3]; /* velocity U of the reference state: populations are
                      stored as g_i = f_i - f0_i(rho0, U).  {0,0,0} gives the
                      rest-state shift f_i - w_i rho0; setting U to the flow's
                      mean (free-stream) velocity keeps the stored values, and
                      their rounding, small.  |U| components <= 0.5; U_z = 0
                      for D2Q9.  Results do not depend on U beyond rounding. */
  double sigma;  /* LBM_HRR only: hybrid weight sigma of eq. a1ij_HRR in
                    [0, 1] (1 = RR; the paper's runs use 0.995); ignored by
                    the other collisions */
} lbm_config;

/* Optional device allocator (e.g. a framework's caching allocator).
 * alloc returns device memory of at least `bytes` bytes aligned to 256 bytes,
 * or NULL on failure; free releases a pointer alloc returned. */
typedef struct {
  void* (*alloc)(size_t bytes, void* user);
  void (*free)(void* ptr, void* user);
  void* user;
} lbm_allocator;

/* Create a run.  Validates the layout:
 *   - every level-l box (l >= 1) must be bounded on at least one axis;
 *   - a bounded axis needs hi - lo >= 4; inside a periodic parent axis,
 *     0 <= lo, hi <= parent count (the box may touch but not cross the
 *     periodic seam) and at least 4 parent cells must stay outside; inside a
 *     bounded parent axis, lo >= 4 and hi <= parent count - 5 (nesting
 *     margin of four parent cells);
 *   - tau0 > 1/2, batch >= 1, (node count along z) x batch <= 65535 and
 *     fewer than 2^31 stored elements (nodes plus padding) per population
 *     plane on every level.
 * `stream` is a cudaStream_t (NULL = legacy default stream).  `alloc` may be
 * NULL.  On success *out receives the handle; on error *out is NULL and no
 * memory is held.  The new run must be initialised with lbm_init on every
 * level and run before lbm_step. */
int lbm_create(const lbm_config* cfg, void* stream, const lbm_allocator* alloc,
               lbm_handle* out);

/* Device bytes lbm_create would allocate for this configuration (level
 * populations and interface histories), computed on the host without
 * touching the device; for admission against a memory budget.  Returns
 * LBM_EINVAL for a layout lbm_create would reject. */
int lbm_bytes(const lbm_config* cfg, unsigned long long* bytes);

/* Level geometry: node counts n[3], relaxation time tau_l, and the number of
 * active nodes (nodes that are updated; the parent nodes strictly inside a
 * child's restriction ring are inactive).  Any output pointer may be NULL. */
int lbm_level_info(lbm_handle h, int level, int* n, double* tau,
                   long long* n_active);

/* Set every node of one level of one run to the equilibrium f^(0)(rho, u)
 * (eq. fEqH; initial populations carry no off-equilibrium part).
 * rho: host [N] doubles; u: host [3][N] doubles (u[2] ignored in 2D).
 * Synchronises on the handle's stream.  The fields are staged in chunks of
 * 4 Mi nodes through two device buffers (at most 256 MB, shared with
 * lbm_macros and kept until lbm_destroy), each chunk's host-to-device copy
 * overlapping the conversion of the previous one; pinned host memory makes
 * the copies run at full speed. */
int lbm_init(lbm_handle h, int level, int run, const double* rho,
             const double* u);

/* Analytic initial states, evaluated in FP64 on the device at every node of
 * every level (node positions in level-0 units, periodic minimum image):
 *   LBM_IC_UNIFORM: rho = rho0 + drho, u = u0;
 *   LBM_IC_VORTEX:  convected vortex of Sec. 10.1 (eq. init_COVO) about the
 *                   z axis through center, with the linearised density
 *                   rho0 [1 - eps^2/(2 cs^2) exp(-r^2/R^2)] and
 *                   u = u0 + eps (-(y-yc), x-xc)/R exp(-r^2/(2R^2));
 *   LBM_IC_PULSE:   Gaussian density pulse of Sec. 9.2 (eq. init_Pulse),
 *                   rho = rho0 [1 + amplitude exp(-r^2/(2R^2))], u = u0. */
#define LBM_IC_UNIFORM 0
#define LBM_IC_VORTEX 1
#define LBM_IC_PULSE 2
typedef struct {
  int kind;
  double u0[3];
  double center[3];
  double radius;    /* R */
  double amplitude; /* pulse amplitude A */
  double eps;       /* vortex strength */
  double drho;      /* uniform density offset */
} lbm_ic;

/* Set every level of one run to the equilibrium of an analytic state
 * (same rules as lbm_init, without host arrays).  Synchronises. */
int lbm_init_analytic(lbm_handle h, int run, const lbm_ic* ic);

/* Advance every run by n_coarse level-0 steps (level l takes 2^l sub-steps
 * each, Sec. 4.3).  Asynchronous.  The first step after lbm_init starts the
 * coarse-to-fine temporal interpolation with the linear rule; later steps
 * use eq. TempInt.  Steps after the first replay captured CUDA graphs unless
 * graphs were switched off with lbm_set_graphs. */
int lbm_step(lbm_handle h, int n_coarse);

/* Use (1, default) or bypass (0) CUDA graphs in lbm_step. */
int lbm_set_graphs(lbm_handle h, int enable);

/* Persistent fused step (mode 1; 0 = off, the default): from the second
 * coarse step on, lbm_step(h, n) issues one cooperative kernel per 1024
 * coarse steps that runs every level update, history capture, rebuild,
 * restriction and probe of those steps in the scheduler's order, separated
 * by grid barriers, instead of one kernel per operation.  Meant for small
 * runs, whose per-operation kernels are dominated by launch and drain
 * time.  Plain, regularized and recursive regularized collisions without
 * sensors (LBM_EINVAL for the hybrid collision; while sensors are on, or
 * while profiling, lbm_step uses the per-operation kernels).  Every
 * barrier wait is bounded (about a second); if one runs out the kernel
 * stops, the run's state is lost, and the next lbm_step or lbm_sync
 * returns LBM_ETIMEOUT until lbm_set_fused is called again.  Mode 2 is a
 * test of that path: its barriers wait for one block more than the launch
 * has and give up after a few milliseconds.  Synchronises. */
int lbm_set_fused(lbm_handle h, int mode);

/* Macroscopic density and velocity of one level of one run, from the
 * post-collision state after the last step: rho host [N], u host [3][N]
 * (u[2] = 0 in 2D); NaN at inactive nodes.  Synchronises.  Converted in
 * chunks through lbm_init's two staging buffers, each chunk's device-to-host
 * copy overlapping the conversion of the next; pinned host memory makes the
 * copies run at full speed. */
int lbm_macros(lbm_handle h, int level, int run, double* rho, double* u);

/* Same as lbm_macros but into device buffers (float): rho_dev [N],
 * u_dev [3][N].  Asynchronous on the handle's stream. */
int lbm_macros_device(lbm_handle h, int level, int run, float* rho_dev,
                      float* u_dev);

/* Post-collision populations of one level of one run, shifted by the rest
 * state (f_i - w_i rho0, whatever u_ref is), host [q][N] doubles, in the
 * library's velocity order (returned by lbm_lattice).  Synchronises; keeps
 * its device buffer like lbm_macros. */
int lbm_populations(lbm_handle h, int level, int run, double* g);

/* The library's velocity set: xi host [q][3] ints, w host [q] doubles.
 * Returns q (> 0) or a negative code. */
int lbm_lattice(int lattice, int* xi, double* w);

/* Register probe nodes: n nodes of `level`, ijk host [n][3] node indices.
 * After every coarse step the density and velocity of each probe of each
 * run are recorded on the device (capacity: min(65536, max(16, 2^26 /
 * (batch * n * 4))) coarse steps; older samples are overwritten).  Replaces
 * any earlier probe set. */
int lbm_probe_add(lbm_handle h, int level, int n, const int* ijk);

/* Drain the probe record: out host [n_steps][batch][n][4] doubles
 * (rho, u_x, u_y, u_z), oldest first, at most max_steps; *n_steps receives
 * the number of recorded steps returned.  Synchronises. */
int lbm_probe(lbm_handle h, double* out, int max_steps, int* n_steps);

/* Asynchronous form of lbm_probe for a loop that reads every step's samples
 * without stalling the device: enqueues, on the handle's stream after the
 * work issued so far, the copies of the newest min(pending, max_steps)
 * recorded steps into out (same layout as lbm_probe) and the reset of the
 * record, and returns at once with that count in *n_steps.  "Pending" is
 * counted on the host: one record per coarse step issued by lbm_step since
 * the last read-out or lbm_probe_add (at most the record's capacity).
 * out is owned by the caller and must stay valid, untouched, until
 * lbm_sync(h) (or any synchronising call) returns; pinned host memory lets
 * the copies overlap the following steps (pageable memory works but the
 * driver may stage the copy synchronously).  Does not allocate. */
int lbm_probe_async(lbm_handle h, double* out, int max_steps, int* n_steps);

/* FP64 conservation diagnostics of one run, reduced on the device in a fixed
 * order (deterministic): per level, mass[l] = sum over active nodes of
 * (rho - rho0) and mom[l][3] = sum of rho u, in level lattice units.
 * Returns LBM_EUNSTABLE if any sum is not finite.  Synchronises. */
int lbm_diag(lbm_handle h, int run, double* mass, double* mom);

/* Same result as lbm_diag, computed without allocating anything.  The paper
 * has no counterpart: this serves callers that cannot let the library
 * allocate device memory -- a serving loop bound to a fixed device-memory
 * budget, a process whose device memory belongs to another framework's
 * pool, or a monitor that cannot take the device-wide synchronisation of
 * cudaFree.  The partial sums live in one fixed device array of 2 MiB inside
 * the library (held by every GPU that loads the library until the process
 * exits).  Limit: every level of the run must have at most 16,777,216 nodes
 * (2^24); a run with a larger level is rejected with LBM_EINVAL before any
 * device work.  Every call must be made with the handle's device current
 * (the device that was current at lbm_create); otherwise it returns
 * LBM_EINVAL before any device work.  The first call on a device looks the
 * array's address up once for that device, so make that first call before
 * any stream capture.  All calls share the one array:
 * calls whose device work overlaps in time (different streams, or several
 * handles at once) race and must be serialised by the caller; nothing in the
 * array needs clearing, because every call writes each value before reading
 * it.  Synchronises. */
int lbm_diag_noalloc(lbm_handle h, int run, double* mass, double* mom);

/* Spurious-noise diagnostic: the density difference between a refined run
 * and the same initial state on the uniform level-0 grid alone (a second
 * handle, `single`, with the same level-0 layout, lattice and storage),
 * over level-0 nodes outside the refined run's level-1 box by at least
 * `margin` cells on every bounded axis, where the refined solution should
 * only differ by what the interface emits.  Reduced in FP64 on the device:
 * *max_abs = max |rho_refined - rho_single|, *rms = root mean square,
 * *count = nodes used (may be NULL).  Synchronises both handles. */
int lbm_noise(lbm_handle refined, lbm_handle single, int run, int margin,
              double* max_abs, double* rms, long long* count);

/* Block until all work issued by the handle has finished. */
int lbm_sync(lbm_handle h);

/* Count of CUDA kernel launches issued by this handle so far (graph
 * replays count every kernel node they contain). */
long long lbm_kernel_launches(lbm_handle h);

/* Launch-shape autotuner.  For every level, times the level update with
 * each candidate block shape (32x4, 32x2, 32x1, 64x2, 64x1, 128x1, 32x3
 * threads along x by rows) on a scratch copy of the level (allocated and
 * freed here, so the run itself is untouched), `reps` even + odd update
 * pairs each after one warm-up pair, and keeps the fastest.  The shape
 * changes which nodes share a block, never a node's arithmetic: results are
 * bitwise the same for every shape.  shapes (may be NULL) receives
 * [nlevels][2] = (bx, by).  The hybrid collision's update keeps 32x4.
 * Synchronises; needs device memory for one level's populations. */
int lbm_autotune(lbm_handle h, int reps, int* shapes);

/* Set one level's update block shape explicitly: bx a multiple of 32,
 * bx * by <= 128.  LBM_EINVAL otherwise.  Synchronises. */
int lbm_set_block_shape(lbm_handle h, int level, int bx, int by);

/* Face buffers of the 3D levels whose x axis is bounded by their box: on
 * (1, the default) or off (0).  On: the coarse -> fine rebuild of the
 * nodes on the two faces normal to x writes their populations into a
 * compact face buffer (whole 32-byte sectors; in the population planes x is
 * the fastest axis, so each of those populations would fill a sector of
 * its own) and the level update reads them from there.  Off: the rebuild
 * writes them into the planes.  Results are bitwise the same either way.
 * Not used by the hybrid collision or on levels with sensors on.
 * Synchronises. */
int lbm_set_face_buffer(lbm_handle h, int enable);


/* Non-hydrodynamic mode sensors of Sec. 7 on one level (all runs), from the
 * next coarse step on: at every iteration of the level, from its
 * pre-collision state at middle nodes (not inactive, not TN, not on a
 * refined level's outer node layer),
 *   bit 0 spuriousAc (eq. sensorSpuriousAc): div u(t-1) * div u(t) < 0,
 *   bit 1 spuriousS (eq. sensorSpuriousS): curl u(t-1) . curl u(t) < 0,
 *         each counted only where both factors exceed eps in magnitude
 *         (eps = 0: the literal sign test, which round-off can trip),
 *   bit 2 spuriousG (eq. sensorSpuriousG): |f1G| > g_threshold and neither
 *         other bit, f1G = f^(1) minus its second-order Hermite projection
 *         (eqs. fneqSplit, reguProceduref1S);
 * div u and curl u by second-order central differences.  The state before
 * the first iteration is zero (no flags).  Allocates the level's velocity
 * planes (D binary32 planes) if the collision does not already have them,
 * plus one plane per div / curl component, one for |f1G| and one byte
 * plane, per run;
 * adds a velocity pass (unless H-RR) and a sensor pass to every iteration
 * of the level.  Calling it again changes eps and g_threshold.  Synchronises.
 * Returns LBM_EINVAL for a negative or non-finite eps or threshold. */
int lbm_sensors_enable(lbm_handle h, int level, double eps, double g_threshold);

/* Latest sensor state of one run on one level, in node order (x fastest):
 * flags [N], div [N], curl [3][N] (z component only in 2D) and |f1G| [N]
 * (the quantity the spuriousG bit thresholds); any output may be NULL.
 * LBM_ESTATE if the sensors of the level are not enabled.  Synchronises. */
int lbm_sensors(lbm_handle h, int level, int run, unsigned char* flags, double* div,
                double* curl, double* gnorm);

/* Per-kernel timing.  lbm_profile(h, 1) clears the record and makes the
 * following lbm_step calls launch eagerly (no graph replay) with a CUDA
 * event pair around every kernel on the handle's stream; lbm_profile(h, 0)
 * stops recording.  Both synchronise. */
int lbm_profile(lbm_handle h, int enable);

/* Sum of the recorded kernel durations (ms) and their count for one kernel
 * kind (0 level update, 1 history capture, 2 coarse-to-fine rebuild,
 * 3 fine-to-coarse restriction, 4 probe sampling, 5 velocity pass (LBM_HRR
 * or sensors), 6 parent strain-rate history and 7 outer-layer collision
 * (LBM_HRR), 8 sensor pass) on one level
 * (-1: all levels; the level is the one updated, or the parent for 1, 3
 * and 6).
 * Synchronises. */
int lbm_profile_read(lbm_handle h, int kind, int level, double* total_ms,
                     long long* count);

/* Release the handle and all device memory it owns. NULL is ignored. */
void lbm_destroy(lbm_handle h);

/* Static description of a return code. */
const char* lbm_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* MLBM_H */
