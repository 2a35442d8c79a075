/*
 * FP64 CPU oracle for the multi-level lattice Boltzmann step of
 * Astoul, Wissocq, Boussuge, Sengissen & Sagaut, "Analysis and reduction of
 * spurious noise generated at grid refinement interfaces with the lattice
 * Boltzmann method" (arXiv 2004.11863).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA library
 * against the paper.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it; the product path never does.  It shares no
 * code, header, table or helper with the CUDA implementation.
 *
 * Everything here is plain IEEE double precision, compiled without FMA
 * contraction, with fixed loop orders: the result is deterministic.
 *
 * Conventions
 *   - lattices: 0 = D2Q9 (velocity order of Sec. 3.1, eq. xi_i),
 *               1 = D3Q19, 2 = D3Q27 (generated from their definitions);
 *   - collisions: 0 = BGK (eq. BGKmodel), 1 = projected regularized (REG,
 *                 eqs. reguProcedure..LBMscheme_reg), 2 = recursive
 *                 regularized (RR, eqs. f1RR, a13RR), 3 = hybrid recursive
 *                 regularized (H-RR, eq. a1ij_HRR; Sec. 4.4 step list);
 *   - a level's nodes are numbered x fastest, then y, then z;
 *   - level 0 is periodic on every axis; level l >= 1 is described by a
 *     closed box [lo, hi] in level l-1 node units.  An axis whose box spans
 *     the whole (periodic) parent axis (hi - lo == parent node count) is a
 *     periodic axis of the child with twice the parent's node count; any
 *     other axis is bounded and holds 2 (hi - lo) + 1 child nodes.
 */
#ifndef MLBM_ORACLE_H
#define MLBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_run orc_run;

/* Lattice tables: xi is [q][3] (z component 0 in 2D), w is [q]. Returns q. */
int orc_lattice(int lattice, int* xi, double* w);

/* Third-order Hermite equilibrium f^(0)(rho, u) (eqs. fEqH, fEqO3). */
void orc_feq(int lattice, double rho, const double* u, double* feq);

/* Second-order off-equilibrium Hermite coefficients a1^(2) (eq. a1Proj):
 * a1[3][3] = sum_i H2_i (f_i - f^(0)_i). */
void orc_a1(int lattice, const double* f, double* a1);

/* One local collision: f_out = post-collision state of f_in (eqs. BGKmodel,
 * LBMscheme_reg with f1RR / reguProceduref1N). */
void orc_collide(int lattice, int collision, double tau, const double* f_in,
                 double* f_out);

/* Hybrid recursive regularized collision (collision 3; Sec. 3.3) with a
 * given strain rate S6 = (xx, yy, zz, xy, xz, yz). */
void orc_collide_hrr(int lattice, double tau, double sigma, const double* f_in,
                     const double* S6, double* f_out);

/* Interface weights, exposed so tests can check them against polynomials.
 * time: value at t+1/2 from values at t-1, t, t+1 (eq. TempInt); first=1
 * selects the linear start-up rule used when t-1 does not exist.
 * space: mid-point value from 4 collinear values at -3/2,-1/2,+1/2,+3/2
 * (eq. spaceInt). filter: weight of neighbour offset (dx,dy,dz) in the
 * restriction filter (eq. filterFneq and its tensor-product 3D form). */
double orc_interp_time(double g_m1, double g_0, double g_p1, int first);
double orc_interp_space(double g_m3, double g_m1, double g_p1, double g_p3);
double orc_filter_weight(int d, int dx, int dy, int dz);

/* A multi-level run.
 *   dims: level-0 node counts (dims[2] = 1 for D2Q9);
 *   boxes: (nlevels-1) x {lo[3], hi[3]}; box k places level k+1 inside k.
 * Returns NULL on an invalid layout. */
orc_run* orc_create(int lattice, int collision, double tau0, double rho0,
                    const int* dims, int nlevels, const int* boxes);
void orc_destroy(orc_run* r);
int orc_level_dims(const orc_run* r, int level, int* n);   /* returns N */
double orc_level_tau(const orc_run* r, int level);
/* node classes: 0 inactive, 1 middle, 2 c->f boundary (TF/IE), 3 f->c (TN) */
void orc_level_classes(const orc_run* r, int level, unsigned char* cls);
/* Set every node of a level to f^(0)(rho, u); rho [N], u [3][N]. */
int orc_init_level(orc_run* r, int level, const double* rho, const double* u);
/* Call once after every level is initialised (seeds the history slots). */
int orc_init_done(orc_run* r);
/* Advance n steps of level 0 (each with 2^l sub-steps of level l). */
int orc_step(orc_run* r, int n);
/* Macroscopic rho [N] and u [3][N] of a level from its post-collision state;
 * NaN at inactive nodes. */
int orc_macros(const orc_run* r, int level, double* rho, double* u);
/* Post-collision populations of a level, [q][N]. */
int orc_populations(const orc_run* r, int level, double* f);
/* Hybrid weight sigma of eq. a1ij_HRR for collision 3 (default 1). */
int orc_set_sigma(orc_run* r, double sigma);
/* Non-hydrodynamic mode sensors of a level (Sec. 7, eqs. sensorSpuriousAc,
 * sensorSpuriousS, sensorSpuriousG), evaluated at every later iteration of
 * the level from its pre-collision state at middle nodes.  eps: the sign
 * tests of the first two count only where both factors exceed eps in
 * magnitude (0 = the paper's literal tests); g_threshold: the spuriousG
 * sensor fires where |f1G| exceeds it (0 = the paper's "> 0").
 * orc_sensors returns the latest flags [N] (bit 0 spuriousAc, bit 1
 * spuriousS, bit 2 spuriousG), div u [N], curl u [3][N] and |f1G| [N] (any
 * may be NULL).  Both return -1 on a bad argument. */
int orc_sensors_enable(orc_run* r, int level, double eps, double g_threshold);
int orc_sensors(const orc_run* r, int level, unsigned char* flags, double* div, double* curl,
                double* gnorm);
/* Set a level's populations directly, f [q][N] (post-collision state). */
int orc_set_populations(orc_run* r, int level, const double* f);
/* Set the worker thread count (0 = OpenMP default); returns the count used. */
int orc_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
