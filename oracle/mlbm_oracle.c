/*
 * FP64 CPU oracle for the multi-level lattice Boltzmann step of arXiv
 * 2004.11863 (Astoul et al.).  TEST INFRASTRUCTURE ONLY: used by the tests,
 * the smoke check and the benchmark's CPU-baseline leg, never by the product
 * path.  It shares no code with the CUDA library.
 *
 * The scheme is written in population space with separate pre- and
 * post-collision arrays and follows the cell-vertex algorithm of Sec. 4.3
 * (Lagrava et al., with the overlap of Fig. Overlap); the hybrid model adds
 * the velocity-gradient transfers of Sec. 4.4.  Per step of level l:
 *   stream the middle nodes of level l;
 *   rebuild the c->f boundary nodes (TF by temporal interpolation, IE by
 *       spatial interpolation) with eq. rescff;
 *   if level l has a finer level: record the pre-collision state of level l
 *       on the finer box surface (coarse history at t+1), run the two finer
 *       sub-steps, then rebuild the f->c nodes (TN) with eqs. filterFneq and
 *       rescfc (the restriction of the synchronous iteration);
 *   collide every active node of level l.
 *
 * Readings taken where the paper is silent or garbled:
 *   - eq. TempInt prints its first point as t-1/2; the weights (-1/8,3/4,3/8)
 *     are the quadratic Lagrange weights through t-1, t, t+1 at t+1/2, so the
 *     point is read as t-1.  On a level's very first step, where t-1 does not
 *     exist, the linear rule (g(t)+g(t+1))/2 is used.
 *   - the history at t = 0 is (rho, u) of the initial state with f^(1) = 0;
 *   - all q populations are rebuilt at TF, IE and TN nodes;
 *   - f^(1) is the pre-collision f - f^(0)(rho, u) of the same node;
 *   - the rescaling factors are literally tau_f/(2 tau_c) and 2 tau_c/tau_f;
 *   - eq. reguProceduref1N is read with H^(2);
 *   - 3D: third-order equilibrium and RR terms use the lattice-supported
 *     third-order Hermite set (D3Q27: six H_aab terms with 1/(2 cs^6) and
 *     H_xyz with 1/cs^6; D3Q19: the orthogonal pairs H_aab +- H_ccb with
 *     1/(2 cs^6) and 1/(6 cs^6)); the filter is [1/4,1/2,1/4] per axis; IE
 *     nodes with two odd indices use the tensor-product cubic.
 *   - velocities are interpolated (not momenta), as Sec. 4.3 states.
 */
#include "mlbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define CS2 (1.0 / 3.0)
#define MAXQ 27
#define MAXLEV 4

/* ------------------------------------------------------------------ */
/* Lattices (Sec. 3.1)                                                 */
/* ------------------------------------------------------------------ */

typedef struct {
  int q, d;
  int xi[MAXQ][3];
  double w[MAXQ];
} lattice_t;

static int build_lattice(int id, lattice_t* L) {
  memset(L, 0, sizeof(*L));
  if (id == 0) {
    /* D2Q9, eqs. xi_i and w_i */
    static const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    static const int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    L->q = 9;
    L->d = 2;
    for (int i = 0; i < 9; ++i) {
      L->xi[i][0] = cx[i];
      L->xi[i][1] = cy[i];
      L->xi[i][2] = 0;
      L->w[i] = (i == 0) ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
    return 9;
  }
  if (id == 1 || id == 2) {
    /* D3Q19: velocities with |xi|^2 <= 2; D3Q27: all of {-1,0,1}^3.
     * Weights by speed class: D3Q19 (1/3, 1/18, 1/36);
     * D3Q27 (8/27, 2/27, 1/54, 1/216). */
    const double w19[3] = {1.0 / 3.0, 1.0 / 18.0, 1.0 / 36.0};
    const double w27[4] = {8.0 / 27.0, 2.0 / 27.0, 1.0 / 54.0, 1.0 / 216.0};
    int q = 0;
    L->d = 3;
    for (int s = 0; s <= 3; ++s) /* speed classes in order */
      for (int z = -1; z <= 1; ++z)
        for (int y = -1; y <= 1; ++y)
          for (int x = -1; x <= 1; ++x) {
            int n2 = x * x + y * y + z * z;
            if (n2 != s) continue;
            if (id == 1 && n2 > 2) continue;
            L->xi[q][0] = x;
            L->xi[q][1] = y;
            L->xi[q][2] = z;
            L->w[q] = (id == 1) ? w19[n2] : w27[n2];
            ++q;
          }
    L->q = q;
    return q;
  }
  return 0;
}

int orc_lattice(int lattice, int* xi, double* w) {
  lattice_t L;
  int q = build_lattice(lattice, &L);
  for (int i = 0; i < q; ++i) {
    for (int a = 0; a < 3; ++a) xi[3 * i + a] = L.xi[i][a];
    w[i] = L.w[i];
  }
  return q;
}

/* ------------------------------------------------------------------ */
/* Hermite expansion (eq. fEqH) and its lattice-supported third order  */
/* ------------------------------------------------------------------ */

static double h2(const int* xi, int a, int b) {
  return (double)(xi[a] * xi[b]) - (a == b ? CS2 : 0.0);
}
/* H^(3)_{aab} = xi_a^2 xi_b - cs^2 xi_b  (a != b) */
static double h3aab(const int* xi, int a, int b) {
  return (double)(xi[a] * xi[a] * xi[b]) - CS2 * (double)xi[b];
}
static double h3xyz(const int* xi) { return (double)(xi[0] * xi[1] * xi[2]); }

/* The third-order part sum over the lattice-supported H^(3) terms,
 * weighted as the projection of a symmetric coefficient tensor a3. */
static double third_order(const lattice_t* L, const int* xi,
                          double a3[3][3][3]) {
  const double cs6 = CS2 * CS2 * CS2;
  double s = 0.0;
  if (L->q == 9) {
    /* eq. fEqO3 / f1RR: H_xxy a_xxy + H_xyy a_xyy, over 2 cs^6 */
    s = (h3aab(xi, 0, 1) * a3[0][0][1] + h3aab(xi, 1, 0) * a3[1][1][0]) /
        (2.0 * cs6);
  } else if (L->q == 27) {
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        if (a != b) s += h3aab(xi, a, b) * a3[a][a][b] / (2.0 * cs6);
    s += h3xyz(xi) * a3[0][1][2] / cs6;
  } else {
    /* D3Q19: for each odd axis b, the two other axes a < c give the
     * orthogonal pair h+ = H_aab + H_ccb, h- = H_aab - H_ccb. */
    for (int b = 0; b < 3; ++b) {
      int a = (b == 0) ? 1 : 0;
      int c = (b == 2) ? 1 : 2;
      double hp = h3aab(xi, a, b) + h3aab(xi, c, b);
      double hm = h3aab(xi, a, b) - h3aab(xi, c, b);
      double mp = a3[a][a][b] + a3[c][c][b];
      double mm = a3[a][a][b] - a3[c][c][b];
      s += hp * mp / (2.0 * cs6) + hm * mm / (6.0 * cs6);
    }
  }
  return s;
}

/* w_i [ a0 + xi.a1/cs^2 + H2:a2/(2 cs^4) + third order(a3) ]  (eq. fEqH) */
static double hermite_sum(const lattice_t* L, int i, double a0,
                          const double* a1v, double a2[3][3],
                          double a3[3][3][3]) {
  const int* xi = L->xi[i];
  double s = a0;
  for (int a = 0; a < 3; ++a) s += (double)xi[a] * a1v[a] / CS2;
  double c2 = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) c2 += h2(xi, a, b) * a2[a][b];
  s += c2 / (2.0 * CS2 * CS2);
  s += third_order(L, xi, a3);
  return L->w[i] * s;
}

static void feq_lat(const lattice_t* L, double rho, const double* u,
                    double* feq) {
  double uu[3] = {u[0], u[1], L->d == 2 ? 0.0 : u[2]};
  double m1[3], m2[3][3], m3[3][3][3];
  for (int a = 0; a < 3; ++a) {
    m1[a] = rho * uu[a];
    for (int b = 0; b < 3; ++b) {
      m2[a][b] = rho * uu[a] * uu[b];
      for (int c = 0; c < 3; ++c) m3[a][b][c] = rho * uu[a] * uu[b] * uu[c];
    }
  }
  for (int i = 0; i < L->q; ++i) feq[i] = hermite_sum(L, i, rho, m1, m2, m3);
}

void orc_feq(int lattice, double rho, const double* u, double* feq) {
  lattice_t L;
  build_lattice(lattice, &L);
  feq_lat(&L, rho, u, feq);
}

static void moments(const lattice_t* L, const double* f, double* rho,
                    double* u) {
  double r = 0.0, j[3] = {0, 0, 0};
  for (int i = 0; i < L->q; ++i) {
    r += f[i];
    for (int a = 0; a < 3; ++a) j[a] += (double)L->xi[i][a] * f[i];
  }
  *rho = r;
  for (int a = 0; a < 3; ++a) u[a] = j[a] / r;
}

static void a1_lat(const lattice_t* L, const double* f, const double* feq,
                   double a1[3][3]) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double s = 0.0;
      for (int i = 0; i < L->q; ++i) s += h2(L->xi[i], a, b) * (f[i] - feq[i]);
      a1[a][b] = s;
    }
}

void orc_a1(int lattice, const double* f, double* a1) {
  lattice_t L;
  build_lattice(lattice, &L);
  double rho, u[3], feq[MAXQ], t[3][3];
  moments(&L, f, &rho, u);
  feq_lat(&L, rho, u, feq);
  a1_lat(&L, f, feq, t);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) a1[3 * a + b] = t[a][b];
}

/* Post-collision state (eq. BGKmodel; eq. LBMscheme_reg with
 * eq. reguProceduref1N for REG and eqs. f1RR, a13RR for RR). */
static void collide_lat(const lattice_t* L, int coll, double tau,
                        const double* f, double* out) {
  double rho, u[3], feq[MAXQ];
  moments(L, f, &rho, u);
  feq_lat(L, rho, u, feq);
  const double om = 1.0 - 1.0 / tau;
  if (coll == 0) {
    for (int i = 0; i < L->q; ++i) out[i] = feq[i] + om * (f[i] - feq[i]);
    return;
  }
  double a1[3][3], a3[3][3][3], zero1[3] = {0, 0, 0};
  a1_lat(L, f, feq, a1);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c)
        a3[a][b][c] = (coll == 2)
                          ? u[a] * a1[b][c] + u[b] * a1[a][c] + u[c] * a1[a][b]
                          : 0.0;
  if (L->d == 2)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        for (int c = 0; c < 3; ++c)
          if (a == 2 || b == 2 || c == 2) a3[a][b][c] = 0.0;
  for (int i = 0; i < L->q; ++i) {
    double f1 = hermite_sum(L, i, 0.0, zero1, a1, a3);
    out[i] = feq[i] + om * f1;
  }
}

/* Hybrid recursive regularized collision (Sec. 3.3, eq. a1ij_HRR): the
 * projected a1^(2) is blended with the finite-difference estimate of
 * eq. stressT, a1 = sigma a1^(2) + (1 - sigma)(-2 tau rho cs^2 S); the
 * third order follows by the recursion of eq. a13RR and the post-collision
 * state by eq. f1RR in eq. LBMscheme_reg.  S6 = (xx, yy, zz, xy, xz, yz). */
static void collide_hrr_lat(const lattice_t* L, double tau, double sigma, const double* f,
                            const double* S6, double* out) {
  double rho, u[3], feq[MAXQ];
  moments(L, f, &rho, u);
  feq_lat(L, rho, u, feq);
  double a1p[3][3], a1[3][3], a3[3][3][3], zero1[3] = {0, 0, 0};
  a1_lat(L, f, feq, a1p);
  const double S[3][3] = {{S6[0], S6[3], S6[4]}, {S6[3], S6[1], S6[5]}, {S6[4], S6[5], S6[2]}};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      a1[a][b] = sigma * a1p[a][b] + (1.0 - sigma) * (-2.0 * tau * rho * CS2 * S[a][b]);
  if (L->d == 2)
    for (int a = 0; a < 3; ++a) a1[a][2] = a1[2][a] = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c) {
        a3[a][b][c] = u[a] * a1[b][c] + u[b] * a1[a][c] + u[c] * a1[a][b];
        if (L->d == 2 && (a == 2 || b == 2 || c == 2)) a3[a][b][c] = 0.0;
      }
  const double om = 1.0 - 1.0 / tau;
  for (int i = 0; i < L->q; ++i) out[i] = feq[i] + om * hermite_sum(L, i, 0.0, zero1, a1, a3);
}

void orc_collide_hrr(int lattice, double tau, double sigma, const double* f_in, const double* S6,
                     double* f_out) {
  lattice_t L;
  build_lattice(lattice, &L);
  collide_hrr_lat(&L, tau, sigma, f_in, S6, f_out);
}

void orc_collide(int lattice, int collision, double tau, const double* f_in,
                 double* f_out) {
  lattice_t L;
  build_lattice(lattice, &L);
  collide_lat(&L, collision, tau, f_in, f_out);
}

/* ------------------------------------------------------------------ */
/* Interface stencils (eqs. TempInt, spaceInt, filterFneq)             */
/* ------------------------------------------------------------------ */

static void time_weights(int first, double* w) {
  if (first) {
    w[0] = 0.0;
    w[1] = 0.5;
    w[2] = 0.5;
  } else {
    w[0] = -1.0 / 8.0;
    w[1] = 3.0 / 4.0;
    w[2] = 3.0 / 8.0;
  }
}

double orc_interp_time(double g_m1, double g_0, double g_p1, int first) {
  double w[3];
  time_weights(first, w);
  return w[0] * g_m1 + w[1] * g_0 + w[2] * g_p1;
}

static const double SPACE_W[4] = {-1.0 / 16.0, 9.0 / 16.0, 9.0 / 16.0,
                                  -1.0 / 16.0};

double orc_interp_space(double g_m3, double g_m1, double g_p1, double g_p3) {
  return SPACE_W[0] * g_m3 + SPACE_W[1] * g_m1 + SPACE_W[2] * g_p1 +
         SPACE_W[3] * g_p3;
}

static double filter1(int o) { return o == 0 ? 0.5 : 0.25; }

double orc_filter_weight(int d, int dx, int dy, int dz) {
  double w = filter1(dx) * filter1(dy);
  if (d == 3) w *= filter1(dz);
  else if (dz != 0) w = 0.0;
  return w;
}

/* ------------------------------------------------------------------ */
/* Levels                                                              */
/* ------------------------------------------------------------------ */

enum { C_INACTIVE = 0, C_MIDDLE = 1, C_BOUND = 2, C_TN = 3 };

typedef struct {
  int n[3];     /* node counts */
  int per[3];   /* periodic axes of this level */
  int boxed[3]; /* (l >= 1) axes bounded by the box */
  int lo[3], hi[3];
  long N;
  double tau;
  double* fpost; /* [N][q] */
  double* fpre;  /* [N][q] */
  unsigned char* cls;
  long nsteps;
  /* History of the parent level on this level's box surface:
   * hidx[parent node] -> k or -1; hist[3][K][nv] with nv = 4 + q:
   * (rho, u_x, u_y, u_z, f^(1)_0..q-1). Slot 2 is the newest. */
  long* hidx;
  double* hist;
  long K;
  /* Hybrid model (collision 3) only: pre-collision velocity per node
   * [N][3]; strain rate each node last collided with [N][6] (xx, yy, zz,
   * xy, xz, yz); strain rate handed to a TN node by the finer level [N][6];
   * parent strain-rate history on this level's box surface [3][K][6]. */
  double* vel;
  double* sused;
  double* sgiven;
  double* hists;
  /* Non-hydrodynamic mode sensors (Sec. 7), when enabled: the latest flags
   * per node (bit 0 spuriousAc, bit 1 spuriousS, bit 2 spuriousG), the
   * velocity divergence [N] and vorticity [N][3] of the latest iteration,
   * and a velocity scratch field [N][3]. */
  int sens_on;
  double sens_eps, sens_thr;
  unsigned char* sflag;
  double* sgn; /* |f1G| [N] */
  double* sdiv;
  double* scurl;
  double* svel;
} level_t;

struct orc_run {
  lattice_t L;
  int lattice, coll, nlev, dim;
  double rho0;
  double sigma; /* hybrid weight of eq. a1ij_HRR (collision 3) */
  level_t lev[MAXLEV];
};

static void strain_fd(const orc_run* r, const level_t* v, int x, int y, int z, double* S6);

static long nid(const level_t* v, int x, int y, int z) {
  return ((long)z * v->n[1] + y) * v->n[0] + x;
}

static int wrap(int x, int n) {
  int r = x % n;
  return r < 0 ? r + n : r;
}

/* Position of parent-level coordinate P relative to the child box's lo,
 * in [-1, n_parent - 2] on periodic parent axes. */
static int rel_coord(const level_t* par, const level_t* ch, int a, int P) {
  int r = P - ch->lo[a];
  if (par->per[a]) {
    r = wrap(r, par->n[a]);
    if (r > ch->hi[a] - ch->lo[a] + 1) r -= par->n[a];
  }
  return r;
}

int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

static void free_level(level_t* v) {
  free(v->sflag);
  free(v->sgn);
  free(v->sdiv);
  free(v->scurl);
  free(v->svel);
  free(v->vel);
  free(v->sused);
  free(v->sgiven);
  free(v->hists);
  free(v->fpost);
  free(v->fpre);
  free(v->cls);
  free(v->hidx);
  free(v->hist);
}

void orc_destroy(orc_run* r) {
  if (!r) return;
  for (int l = 0; l < r->nlev; ++l) free_level(&r->lev[l]);
  free(r);
}

/* Classes of level l's nodes with respect to its child (TN, inactive). */
static void mark_child_footprint(orc_run* r, int l) {
  level_t* p = &r->lev[l];
  level_t* c = &r->lev[l + 1];
  for (int z = 0; z < p->n[2]; ++z)
    for (int y = 0; y < p->n[1]; ++y)
      for (int x = 0; x < p->n[0]; ++x) {
        int P[3] = {x, y, z};
        int inside_shrunk = 1, strictly = 1, any_box = 0;
        for (int a = 0; a < r->dim; ++a) {
          if (!c->boxed[a]) continue;
          any_box = 1;
          int E = c->hi[a] - c->lo[a];
          int q = rel_coord(p, c, a, P[a]);
          if (q < 1 || q > E - 1) inside_shrunk = 0;
          if (q < 2 || q > E - 2) strictly = 0;
        }
        if (!any_box) continue;
        long id = nid(p, x, y, z);
        if (strictly)
          p->cls[id] = C_INACTIVE;
        else if (inside_shrunk)
          p->cls[id] = C_TN;
      }
}

/* History map: parent nodes on the child box surface, extended by one
 * parent cell past its edges (needed by the 4-point spatial stencil). */
static int build_history(orc_run* r, int l) {
  level_t* p = &r->lev[l];
  level_t* c = &r->lev[l + 1];
  c->hidx = (long*)malloc(sizeof(long) * p->N);
  if (!c->hidx) return -1;
  long K = 0;
  for (int z = 0; z < p->n[2]; ++z)
    for (int y = 0; y < p->n[1]; ++y)
      for (int x = 0; x < p->n[0]; ++x) {
        int P[3] = {x, y, z};
        int on_face = 0, in_ext = 1;
        for (int a = 0; a < r->dim; ++a) {
          if (!c->boxed[a]) continue;
          int E = c->hi[a] - c->lo[a];
          int q = rel_coord(p, c, a, P[a]);
          if (q == 0 || q == E) on_face = 1;
          if (q < -1 || q > E + 1) in_ext = 0;
        }
        long id = nid(p, x, y, z);
        c->hidx[id] = (on_face && in_ext) ? K++ : -1;
      }
  c->K = K;
  c->hist = (double*)calloc((size_t)3 * K * (4 + r->L.q), sizeof(double));
  return c->hist ? 0 : -1;
}

orc_run* orc_create(int lattice, int collision, double tau0, double rho0,
                    const int* dims, int nlevels, const int* boxes) {
  if (nlevels < 1 || nlevels > MAXLEV) return NULL;
  if (collision < 0 || collision > 3) return NULL;
  if (!(tau0 > 0.5)) return NULL;
  orc_run* r = (orc_run*)calloc(1, sizeof(orc_run));
  if (!r) return NULL;
  if (!build_lattice(lattice, &r->L)) {
    free(r);
    return NULL;
  }
  r->lattice = lattice;
  r->coll = collision;
  r->nlev = nlevels;
  r->dim = r->L.d;
  r->rho0 = rho0;
  r->sigma = 1.0;
  for (int l = 0; l < nlevels; ++l) {
    level_t* v = &r->lev[l];
    if (l == 0) {
      for (int a = 0; a < 3; ++a) {
        v->n[a] = (a < r->dim) ? dims[a] : 1;
        v->per[a] = 1;
        v->boxed[a] = 0;
        if (v->n[a] < 1) goto fail;
      }
      v->tau = tau0;
    } else {
      level_t* p = &r->lev[l - 1];
      const int* b = boxes + 6 * (l - 1);
      for (int a = 0; a < 3; ++a) {
        v->lo[a] = b[a];
        v->hi[a] = b[3 + a];
        if (a >= r->dim) {
          v->n[a] = 1;
          v->per[a] = 1;
          v->boxed[a] = 0;
          continue;
        }
        int E = v->hi[a] - v->lo[a];
        if (p->per[a] && v->lo[a] == 0 && E == p->n[a]) {
          v->boxed[a] = 0;
          v->per[a] = 1;
          v->n[a] = 2 * p->n[a];
        } else {
          if (E < 4) goto fail;
          if (p->per[a]) {
            if (v->lo[a] < 0 || v->lo[a] >= p->n[a]) goto fail;
            if (p->n[a] - E < 4) goto fail;
          } else {
            /* nesting margin of at least 4 parent cells */
            if (v->lo[a] < 4 || v->hi[a] > p->n[a] - 5) goto fail;
          }
          v->boxed[a] = 1;
          v->per[a] = 0;
          v->n[a] = 2 * E + 1;
        }
      }
      /* eq. rescTau: tau_f = 2 tau_c - 1/2 */
      v->tau = 2.0 * p->tau - 0.5;
    }
    v->N = (long)v->n[0] * v->n[1] * v->n[2];
    v->fpost = (double*)calloc((size_t)v->N * r->L.q, sizeof(double));
    v->fpre = (double*)calloc((size_t)v->N * r->L.q, sizeof(double));
    v->cls = (unsigned char*)malloc((size_t)v->N);
    if (!v->fpost || !v->fpre || !v->cls) goto fail;
    if (collision == 3) {
      v->vel = (double*)calloc((size_t)v->N * 3, sizeof(double));
      v->sused = (double*)calloc((size_t)v->N * 6, sizeof(double));
      v->sgiven = (double*)calloc((size_t)v->N * 6, sizeof(double));
      if (!v->vel || !v->sused || !v->sgiven) goto fail;
    }
    /* base classes: boundary layer of a refined level, middle otherwise */
    for (int z = 0; z < v->n[2]; ++z)
      for (int y = 0; y < v->n[1]; ++y)
        for (int x = 0; x < v->n[0]; ++x) {
          int X[3] = {x, y, z};
          int bnd = 0;
          for (int a = 0; a < r->dim; ++a)
            if (v->boxed[a] && (X[a] == 0 || X[a] == v->n[a] - 1)) bnd = 1;
          v->cls[nid(v, x, y, z)] = bnd ? C_BOUND : C_MIDDLE;
        }
  }
  for (int l = 0; l + 1 < nlevels; ++l) {
    int any = 0;
    for (int a = 0; a < r->dim; ++a) any |= r->lev[l + 1].boxed[a];
    if (!any) goto fail; /* a child must be bounded on some axis */
    mark_child_footprint(r, l);
    if (build_history(r, l)) goto fail;
    if (collision == 3) {
      level_t* c = &r->lev[l + 1];
      c->hists = (double*)calloc((size_t)3 * c->K * 6, sizeof(double));
      if (!c->hists) goto fail;
    }
  }
  return r;
fail:
  orc_destroy(r);
  return NULL;
}

int orc_level_dims(const orc_run* r, int level, int* n) {
  if (level < 0 || level >= r->nlev) return -1;
  for (int a = 0; a < 3; ++a) n[a] = r->lev[level].n[a];
  return (int)r->lev[level].N;
}

double orc_level_tau(const orc_run* r, int level) {
  return r->lev[level].tau;
}

void orc_level_classes(const orc_run* r, int level, unsigned char* cls) {
  memcpy(cls, r->lev[level].cls, (size_t)r->lev[level].N);
}

int orc_init_level(orc_run* r, int level, const double* rho, const double* u) {
  if (level < 0 || level >= r->nlev) return -1;
  level_t* v = &r->lev[level];
  const int q = r->L.q;
#pragma omp parallel for schedule(static)
  for (long id = 0; id < v->N; ++id) {
    double uu[3] = {u[id], u[v->N + id], u[2 * v->N + id]};
    feq_lat(&r->L, rho[id], uu, v->fpost + id * q);
    memcpy(v->fpre + id * q, v->fpost + id * q, sizeof(double) * q);
  }
  v->nsteps = 0;
  return 0;
}

int orc_init_done(orc_run* r) {
  const int q = r->L.q, nv = 4 + q;
  for (int l = 0; l + 1 < r->nlev; ++l) {
    level_t* p = &r->lev[l];
    level_t* c = &r->lev[l + 1];
    for (long id = 0; id < p->N; ++id) {
      long k = c->hidx[id];
      if (k < 0) continue;
      double rho, u[3];
      moments(&r->L, p->fpost + id * q, &rho, u);
      for (int s = 1; s <= 2; ++s) {
        double* h = c->hist + ((size_t)s * c->K + k) * nv;
        h[0] = rho;
        h[1] = u[0];
        h[2] = u[1];
        h[3] = u[2];
        for (int i = 0; i < q; ++i) h[4 + i] = 0.0;
      }
    }
  }
  if (r->coll == 3) {
    /* strain-rate history at t = 0 from the initial velocity field */
    for (int l = 0; l < r->nlev; ++l) {
      level_t* v = &r->lev[l];
      for (long id = 0; id < v->N; ++id) {
        double rho, u[3];
        moments(&r->L, v->fpost + id * q, &rho, u);
        for (int a = 0; a < 3; ++a) v->vel[id * 3 + a] = u[a];
      }
    }
    for (int l = 0; l + 1 < r->nlev; ++l) {
      level_t* p = &r->lev[l];
      level_t* c = &r->lev[l + 1];
      for (int z = 0; z < p->n[2]; ++z)
        for (int y = 0; y < p->n[1]; ++y)
          for (int x = 0; x < p->n[0]; ++x) {
            long k = c->hidx[nid(p, x, y, z)];
            if (k < 0) continue;
            double S6[6];
            strain_fd(r, p, x, y, z, S6);
            for (int sl = 1; sl <= 2; ++sl)
              memcpy(c->hists + ((size_t)sl * c->K + k) * 6, S6, sizeof(S6));
          }
    }
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* One step of level l (recursive)                                     */
/* ------------------------------------------------------------------ */

static void stream_level(orc_run* r, level_t* v) {
  const lattice_t* L = &r->L;
  const int q = L->q;
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < v->n[2]; ++z)
    for (int y = 0; y < v->n[1]; ++y)
      for (int x = 0; x < v->n[0]; ++x) {
        long id = nid(v, x, y, z);
        if (v->cls[id] != C_MIDDLE) continue;
        for (int i = 0; i < q; ++i) {
          int s[3] = {x - L->xi[i][0], y - L->xi[i][1], z - L->xi[i][2]};
          for (int a = 0; a < 3; ++a)
            if (v->per[a]) s[a] = wrap(s[a], v->n[a]);
          v->fpre[id * q + i] = v->fpost[nid(v, s[0], s[1], s[2]) * q + i];
        }
      }
}

/* Parent coordinate of a child index on axis a (even child index). */
static int parent_coord(const level_t* p, const level_t* c, int a, int x) {
  int P = c->boxed[a] ? c->lo[a] + x / 2 : x / 2;
  if (p->per[a]) P = wrap(P, p->n[a]);
  return P;
}

/* Temporally interpolated (rho, u, f1) of parent node P into g[nv]. */
static void hist_at(const orc_run* r, const level_t* p, const level_t* c,
                    const int* P, const double* wt, double* g) {
  const int nv = 4 + r->L.q;
  long k = c->hidx[nid(p, P[0], P[1], P[2])];
  if (k < 0) abort(); /* layout error: stencil left the history band */
  for (int j = 0; j < nv; ++j) {
    double s = 0.0;
    for (int t = 0; t < 3; ++t)
      s += wt[t] * c->hist[((size_t)t * c->K + k) * nv + j];
    g[j] = s;
  }
}

/* Asynchronous fine sub-step (wt = temporal weights) or synchronous one
 * (wt = {0,0,1}):
 * rebuild every TF/IE node of level l from the parent history. */
static void rebuild_boundary(orc_run* r, int l, const double* wt) {
  level_t* c = &r->lev[l];
  const level_t* p = &r->lev[l - 1];
  const lattice_t* L = &r->L;
  const int q = L->q, nv = 4 + q;
  const double resc = c->tau / (2.0 * p->tau); /* eq. rescff */
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < c->n[2]; ++z)
    for (int y = 0; y < c->n[1]; ++y)
      for (int x = 0; x < c->n[0]; ++x) {
        long id = nid(c, x, y, z);
        if (c->cls[id] != C_BOUND) continue;
        int X[3] = {x, y, z};
        int odd[2], nodd = 0;
        for (int a = 0; a < r->dim; ++a)
          if (X[a] & 1) odd[nodd++] = a;
        double g[4 + MAXQ], acc[4 + MAXQ];
        for (int j = 0; j < nv; ++j) acc[j] = 0.0;
        /* nodd = 0: TF, co-located (eq. TempInt or direct transfer);
         * nodd = 1: IE, 4-point cubic along the odd axis (eq. spaceInt);
         * nodd = 2: IE at a face centre, tensor product of two cubics. */
        int n0 = nodd >= 1 ? 4 : 1, n1 = nodd >= 2 ? 4 : 1;
        for (int s0 = 0; s0 < n0; ++s0)
          for (int s1 = 0; s1 < n1; ++s1) {
            int Xc[3] = {X[0], X[1], X[2]};
            double w = 1.0;
            if (nodd >= 1) {
              Xc[odd[0]] = X[odd[0]] - 3 + 2 * s0;
              w *= SPACE_W[s0];
            }
            if (nodd >= 2) {
              Xc[odd[1]] = X[odd[1]] - 3 + 2 * s1;
              w *= SPACE_W[s1];
            }
            int P[3];
            for (int a = 0; a < 3; ++a)
              P[a] = (a < r->dim) ? parent_coord(p, c, a, Xc[a]) : 0;
            hist_at(r, p, c, P, wt, g);
            for (int j = 0; j < nv; ++j) acc[j] += w * g[j];
          }
        double feq[MAXQ];
        feq_lat(L, acc[0], acc + 1, feq);
        for (int i = 0; i < q; ++i)
          c->fpre[id * q + i] = feq[i] + resc * acc[4 + i];
      }
}

/* Record the parent's pre-collision (rho, u, f^(1)) at t+1 on the child
 * box surface, shifting the older slots down (Sec. 4.3, before the fine
 * sub-steps). */
static void capture_history(orc_run* r, int l) {
  level_t* p = &r->lev[l];
  level_t* c = &r->lev[l + 1];
  const lattice_t* L = &r->L;
  const int q = L->q, nv = 4 + q;
  for (long id = 0; id < p->N; ++id) {
    long k = c->hidx[id];
    if (k < 0) continue;
    double* h0 = c->hist + ((size_t)0 * c->K + k) * nv;
    double* h1 = c->hist + ((size_t)1 * c->K + k) * nv;
    double* h2s = c->hist + ((size_t)2 * c->K + k) * nv;
    memcpy(h0, h1, sizeof(double) * nv);
    memcpy(h1, h2s, sizeof(double) * nv);
    const double* f = p->fpre + id * q;
    double rho, u[3], feq[MAXQ];
    moments(L, f, &rho, u);
    feq_lat(L, rho, u, feq);
    h2s[0] = rho;
    h2s[1] = u[0];
    h2s[2] = u[1];
    h2s[3] = u[2];
    for (int i = 0; i < q; ++i) h2s[4 + i] = f[i] - feq[i];
  }
}

/* Restriction: filter the child's pre-collision f^(1) around the node
 * co-located with each TN node (eq. filterFneq) and rebuild the TN node
 * with eq. rescfc from the co-located child node's rho and u. */
static void restrict_tn(orc_run* r, int l) {
  level_t* p = &r->lev[l];
  const level_t* c = &r->lev[l + 1];
  const lattice_t* L = &r->L;
  const int q = L->q, D = r->dim;
  const double resc = 2.0 * p->tau / c->tau;
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < p->n[2]; ++z)
    for (int y = 0; y < p->n[1]; ++y)
      for (int x = 0; x < p->n[0]; ++x) {
        long id = nid(p, x, y, z);
        if (p->cls[id] != C_TN) continue;
        int P[3] = {x, y, z}, X[3] = {0, 0, 0};
        for (int a = 0; a < D; ++a)
          X[a] = c->boxed[a] ? 2 * rel_coord(p, c, a, P[a]) : 2 * P[a];
        double f1s[MAXQ], rho_c = 0, u_c[3] = {0, 0, 0};
        for (int i = 0; i < q; ++i) f1s[i] = 0.0;
        int dzr = (D == 3) ? 1 : 0;
        for (int dz = -dzr; dz <= dzr; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              int s[3] = {X[0] + dx, X[1] + dy, X[2] + dz};
              for (int a = 0; a < 3; ++a)
                if (c->per[a]) s[a] = wrap(s[a], c->n[a]);
              const double* f = c->fpre + nid(c, s[0], s[1], s[2]) * q;
              double rho, u[3], feq[MAXQ];
              moments(L, f, &rho, u);
              feq_lat(L, rho, u, feq);
              double w = orc_filter_weight(D, dx, dy, dz);
              for (int i = 0; i < q; ++i) f1s[i] += w * (f[i] - feq[i]);
              if (dx == 0 && dy == 0 && dz == 0) {
                rho_c = rho;
                u_c[0] = u[0];
                u_c[1] = u[1];
                u_c[2] = u[2];
              }
            }
        double feq[MAXQ];
        feq_lat(L, rho_c, u_c, feq);
        for (int i = 0; i < q; ++i) p->fpre[id * q + i] = feq[i] + resc * f1s[i];
      }
}

static void collide_level(orc_run* r, level_t* v) {
  const int q = r->L.q;
#pragma omp parallel for schedule(static)
  for (long id = 0; id < v->N; ++id) {
    if (v->cls[id] == C_INACTIVE) continue;
    collide_lat(&r->L, r->coll, v->tau, v->fpre + id * q, v->fpost + id * q);
  }
}

/* ---------------- hybrid model (collision 3): Sec. 4.4 ------------------ */

/* Pre-collision velocity of every active node of a level. */
static void velocity_field(orc_run* r, level_t* v) {
  const int q = r->L.q;
#pragma omp parallel for schedule(static)
  for (long id = 0; id < v->N; ++id) {
    if (v->cls[id] == C_INACTIVE) continue;
    double rho, u[3];
    moments(&r->L, v->fpre + id * q, &rho, u);
    for (int a = 0; a < 3; ++a) v->vel[id * 3 + a] = u[a];
  }
}

/* Second-order central differences of the velocity field:
 * S_ab = (d_a u_b + d_b u_a) / 2, d_a u ~ (u(x+e_a) - u(x-e_a)) / 2. */
static void strain_fd(const orc_run* r, const level_t* v, int x, int y, int z, double* S6) {
  double g[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}; /* g[a][b] = d_a u_b */
  const int X[3] = {x, y, z};
  for (int a = 0; a < r->dim; ++a) {
    int P[3] = {X[0], X[1], X[2]}, M[3] = {X[0], X[1], X[2]};
    P[a] += 1;
    M[a] -= 1;
    if (v->per[a]) {
      P[a] = wrap(P[a], v->n[a]);
      M[a] = wrap(M[a], v->n[a]);
    }
    const double* up = v->vel + nid(v, P[0], P[1], P[2]) * 3;
    const double* um = v->vel + nid(v, M[0], M[1], M[2]) * 3;
    for (int b = 0; b < 3; ++b) g[a][b] = 0.5 * (up[b] - um[b]);
  }
  S6[0] = g[0][0];
  S6[1] = g[1][1];
  S6[2] = g[2][2];
  S6[3] = 0.5 * (g[0][1] + g[1][0]);
  S6[4] = 0.5 * (g[0][2] + g[2][0]);
  S6[5] = 0.5 * (g[1][2] + g[2][1]);
}

/* Collide the middle and TN nodes of a level: S from finite differences,
 * or, at TN nodes, the strain rate handed down by the finer level after the
 * restriction (Sec. 4.4, synchronous iteration). */
static void collide_interior_hrr(orc_run* r, level_t* v) {
  const int q = r->L.q;
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < v->n[2]; ++z)
    for (int y = 0; y < v->n[1]; ++y)
      for (int x = 0; x < v->n[0]; ++x) {
        long id = nid(v, x, y, z);
        if (v->cls[id] != C_MIDDLE && v->cls[id] != C_TN) continue;
        double S6[6];
        if (v->cls[id] == C_TN)
          memcpy(S6, v->sgiven + id * 6, sizeof(S6));
        else
          strain_fd(r, v, x, y, z, S6);
        memcpy(v->sused + id * 6, S6, sizeof(S6));
        collide_hrr_lat(&r->L, v->tau, r->sigma, v->fpre + id * q, S6, v->fpost + id * q);
      }
}

/* Sec. 4.4, asynchronous iteration, after the fine middle collision: the
 * parent velocity at its TN nodes at t+1 from a fictitious streaming of the
 * child's post-collision state over the co-located child node's
 * neighbours, then the parent strain rate at t+1 on the child box surface
 * by finite differences, stored as the newest strain-rate history slot. */
static void parent_strain(orc_run* r, int l) {
  level_t* p = &r->lev[l];
  level_t* c = &r->lev[l + 1];
  const lattice_t* L = &r->L;
  const int q = L->q;
  for (int z = 0; z < p->n[2]; ++z)
    for (int y = 0; y < p->n[1]; ++y)
      for (int x = 0; x < p->n[0]; ++x) {
        long id = nid(p, x, y, z);
        if (p->cls[id] != C_TN) continue;
        int P[3] = {x, y, z}, X[3] = {0, 0, 0};
        for (int a = 0; a < r->dim; ++a)
          X[a] = c->boxed[a] ? 2 * rel_coord(p, c, a, P[a]) : 2 * P[a];
        double f[MAXQ], rho, u[3];
        for (int i = 0; i < q; ++i) {
          int s[3] = {X[0] - L->xi[i][0], X[1] - L->xi[i][1], X[2] - L->xi[i][2]};
          for (int a = 0; a < 3; ++a)
            if (c->per[a]) s[a] = wrap(s[a], c->n[a]);
          f[i] = c->fpost[nid(c, s[0], s[1], s[2]) * q + i];
        }
        moments(L, f, &rho, u);
        for (int a = 0; a < 3; ++a) p->vel[id * 3 + a] = u[a];
      }
  for (int z = 0; z < p->n[2]; ++z)
    for (int y = 0; y < p->n[1]; ++y)
      for (int x = 0; x < p->n[0]; ++x) {
        long id = nid(p, x, y, z);
        long k = c->hidx[id];
        if (k < 0) continue;
        strain_fd(r, p, x, y, z, c->hists + ((size_t)2 * c->K + k) * 6);
      }
}

/* Sec. 4.4, both fine sub-steps: the boundary nodes of a child level take
 * the parent strain rate, interpolated in time (eq. TempInt) and space
 * (eq. spaceInt) like the populations, rescaled by eq. PijResc
 * (S^f = S^c / 2), and collide with it. */
static void collide_boundary_hrr(orc_run* r, int l, const double* wt) {
  level_t* c = &r->lev[l];
  const level_t* p = &r->lev[l - 1];
  const int q = r->L.q;
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < c->n[2]; ++z)
    for (int y = 0; y < c->n[1]; ++y)
      for (int x = 0; x < c->n[0]; ++x) {
        long id = nid(c, x, y, z);
        if (c->cls[id] != C_BOUND) continue;
        int X[3] = {x, y, z};
        int odd[2], nodd = 0;
        for (int a = 0; a < r->dim; ++a)
          if (X[a] & 1) odd[nodd++] = a;
        double S6[6] = {0, 0, 0, 0, 0, 0};
        int n0 = nodd >= 1 ? 4 : 1, n1 = nodd >= 2 ? 4 : 1;
        for (int s0 = 0; s0 < n0; ++s0)
          for (int s1 = 0; s1 < n1; ++s1) {
            int Xc[3] = {X[0], X[1], X[2]};
            double w = 1.0;
            if (nodd >= 1) {
              Xc[odd[0]] = X[odd[0]] - 3 + 2 * s0;
              w *= SPACE_W[s0];
            }
            if (nodd >= 2) {
              Xc[odd[1]] = X[odd[1]] - 3 + 2 * s1;
              w *= SPACE_W[s1];
            }
            int P[3];
            for (int a = 0; a < 3; ++a)
              P[a] = (a < r->dim) ? parent_coord(p, c, a, Xc[a]) : 0;
            long k = c->hidx[nid(p, P[0], P[1], P[2])];
            if (k < 0) abort();
            for (int j = 0; j < 6; ++j) {
              double v = 0.0;
              for (int t = 0; t < 3; ++t) v += wt[t] * c->hists[((size_t)t * c->K + k) * 6 + j];
              S6[j] += w * v;
            }
          }
        for (int j = 0; j < 6; ++j) S6[j] *= 0.5; /* eq. PijResc */
        memcpy(c->sused + id * 6, S6, sizeof(S6));
        collide_hrr_lat(&r->L, c->tau, r->sigma, c->fpre + id * q, S6, c->fpost + id * q);
      }
}

/* ---------------- non-hydrodynamic mode sensors (Sec. 7) ----------------- */

/* Central-difference velocity gradient g[a][b] = d_a u_b of a [N][3] field. */
static void grad_fd(const orc_run* r, const level_t* v, const double* field, int x, int y, int z,
                    double g[3][3]) {
  const int X[3] = {x, y, z};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) g[a][b] = 0.0;
  for (int a = 0; a < r->dim; ++a) {
    int P[3] = {X[0], X[1], X[2]}, M[3] = {X[0], X[1], X[2]};
    P[a] += 1;
    M[a] -= 1;
    if (v->per[a]) {
      P[a] = wrap(P[a], v->n[a]);
      M[a] = wrap(M[a], v->n[a]);
    }
    const double* up = field + nid(v, P[0], P[1], P[2]) * 3;
    const double* um = field + nid(v, M[0], M[1], M[2]) * 3;
    for (int b = 0; b < 3; ++b) g[a][b] = 0.5 * (up[b] - um[b]);
  }
}

/* Evaluate the three sensors of one iteration of a level from its
 * pre-collision state (call once every active node's pre-collision state
 * is final, just before the collision):
 *   spuriousAc (eq. sensorSpuriousAc): div u(t-1) * div u(t) < 0;
 *   spuriousS (eq. sensorSpuriousS): curl u(t-1) . curl u(t) < 0;
 *   (both only where each factor's magnitude exceeds eps: at round-off
 *   level the sign is noise; eps = 0 is the literal test)
 *   spuriousG (eq. sensorSpuriousG): |f1G| > threshold and neither of the
 *     two others, with f1 = f - f^(0)(rho, u) split as eq. fneqSplit into
 *     its projection on the second-order Hermite polynomials
 *     (eq. reguProceduref1S, w_i / (2 cs^4) H2_i : a1) and the rest f1G.
 * Evaluated at middle nodes (the central differences need active
 * neighbours); other nodes get no flags.  div and curl of the previous
 * iteration are zero before the first evaluation. */
static void sensors_level(orc_run* r, level_t* v) {
  if (!v->sens_on) return;
  const lattice_t* L = &r->L;
  const int q = L->q;
#pragma omp parallel for schedule(static)
  for (long id = 0; id < v->N; ++id) {
    double rho, u[3] = {0, 0, 0};
    if (v->cls[id] != 0) moments(L, v->fpre + id * q, &rho, u);
    for (int a = 0; a < 3; ++a) v->svel[id * 3 + a] = u[a];
  }
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < v->n[2]; ++z)
    for (int y = 0; y < v->n[1]; ++y)
      for (int x = 0; x < v->n[0]; ++x) {
        const long id = nid(v, x, y, z);
        double* cu = v->scurl + id * 3;
        if (v->cls[id] != C_MIDDLE) {
          v->sflag[id] = 0;
          v->sgn[id] = 0.0;
          v->sdiv[id] = 0.0;
          cu[0] = cu[1] = cu[2] = 0.0;
          continue;
        }
        double g[3][3];
        grad_fd(r, v, v->svel, x, y, z, g);
        const double div = g[0][0] + g[1][1] + g[2][2];
        const double curl[3] = {g[1][2] - g[2][1], g[2][0] - g[0][2], g[0][1] - g[1][0]};
        const double eps = v->sens_eps;
        const double nc0 = sqrt(cu[0] * cu[0] + cu[1] * cu[1] + cu[2] * cu[2]);
        const double nc1 = sqrt(curl[0] * curl[0] + curl[1] * curl[1] + curl[2] * curl[2]);
        const int ac = v->sdiv[id] * div < 0.0 && fabs(v->sdiv[id]) > eps && fabs(div) > eps;
        const int sh = cu[0] * curl[0] + cu[1] * curl[1] + cu[2] * curl[2] < 0.0 && nc0 > eps &&
                       nc1 > eps;
        /* ghost part of the off-equilibrium populations */
        const double* f = v->fpre + id * q;
        double rho, uu[3], feq[MAXQ], a1[3][3];
        moments(L, f, &rho, uu);
        feq_lat(L, rho, uu, feq);
        a1_lat(L, f, feq, a1);
        double n2 = 0.0;
        for (int i = 0; i < q; ++i) {
          double h = 0.0;
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) h += h2(L->xi[i], a, b) * a1[a][b];
          const double f1s = L->w[i] / (2.0 * CS2 * CS2) * h;
          const double f1g = (f[i] - feq[i]) - f1s;
          n2 += f1g * f1g;
        }
        const int gh = sqrt(n2) > v->sens_thr && !ac && !sh;
        v->sflag[id] = (unsigned char)(ac | (sh << 1) | (gh << 2));
        v->sgn[id] = sqrt(n2);
        v->sdiv[id] = div;
        for (int a = 0; a < 3; ++a) cu[a] = curl[a];
      }
}

int orc_sensors_enable(orc_run* r, int level, double eps, double g_threshold) {
  if (level < 0 || level >= r->nlev || !(g_threshold >= 0.0) || !(eps >= 0.0)) return -1;
  level_t* v = &r->lev[level];
  if (!v->sens_on) {
    v->sflag = (unsigned char*)calloc((size_t)v->N, 1);
    v->sgn = (double*)calloc((size_t)v->N, sizeof(double));
    v->sdiv = (double*)calloc((size_t)v->N, sizeof(double));
    v->scurl = (double*)calloc((size_t)v->N * 3, sizeof(double));
    v->svel = (double*)calloc((size_t)v->N * 3, sizeof(double));
    if (!v->sflag || !v->sgn || !v->sdiv || !v->scurl || !v->svel) return -1;
  }
  v->sens_on = 1;
  v->sens_eps = eps;
  v->sens_thr = g_threshold;
  return 0;
}

int orc_sensors(const orc_run* r, int level, unsigned char* flags, double* div, double* curl,
                double* gnorm) {
  if (level < 0 || level >= r->nlev) return -1;
  const level_t* v = &r->lev[level];
  if (!v->sens_on) return -1;
  for (long id = 0; id < v->N; ++id) {
    if (flags) flags[id] = v->sflag[id];
    if (div) div[id] = v->sdiv[id];
    if (gnorm) gnorm[id] = v->sgn[id];
    if (curl)
      for (int a = 0; a < 3; ++a) curl[(size_t)a * v->N + id] = v->scurl[id * 3 + a];
  }
  return 0;
}

int orc_set_populations(orc_run* r, int level, const double* f) {
  if (level < 0 || level >= r->nlev) return -1;
  level_t* v = &r->lev[level];
  const int q = r->L.q;
  for (long id = 0; id < v->N; ++id)
    for (int i = 0; i < q; ++i) {
      v->fpost[id * q + i] = f[(size_t)i * v->N + id];
      v->fpre[id * q + i] = v->fpost[id * q + i];
    }
  v->nsteps = 0;
  return 0;
}

static void advance_hrr(orc_run* r, int l, const double* wt, int first_substep) {
  level_t* v = &r->lev[l];
  stream_level(r, v);
  if (l >= 1) rebuild_boundary(r, l, wt);
  velocity_field(r, v);
  if (l + 1 < r->nlev) {
    level_t* c = &r->lev[l + 1];
    capture_history(r, l);
    memcpy(c->hists, c->hists + (size_t)c->K * 6, sizeof(double) * c->K * 6);
    memcpy(c->hists + (size_t)c->K * 6, c->hists + (size_t)2 * c->K * 6,
           sizeof(double) * c->K * 6);
    double wA[3], wB[3] = {0.0, 0.0, 1.0};
    time_weights(v->nsteps == 0, wA);
    advance_hrr(r, l + 1, wA, 1);
    advance_hrr(r, l + 1, wB, 0);
    restrict_tn(r, l);
    /* TN nodes: velocity of the rebuilt state, strain rate 2 S^f of the
     * co-located child node (eq. PijResc) */
    const int q = r->L.q;
    for (int z = 0; z < v->n[2]; ++z)
      for (int y = 0; y < v->n[1]; ++y)
        for (int x = 0; x < v->n[0]; ++x) {
          long id = nid(v, x, y, z);
          if (v->cls[id] != C_TN) continue;
          double rho, u[3];
          moments(&r->L, v->fpre + id * q, &rho, u);
          for (int a = 0; a < 3; ++a) v->vel[id * 3 + a] = u[a];
          int P[3] = {x, y, z}, X[3] = {0, 0, 0};
          for (int a = 0; a < r->dim; ++a)
            X[a] = c->boxed[a] ? 2 * rel_coord(v, c, a, P[a]) : 2 * P[a];
          const double* sf = c->sused + nid(c, X[0], X[1], X[2]) * 6;
          for (int j = 0; j < 6; ++j) v->sgiven[id * 6 + j] = 2.0 * sf[j];
        }
  }
  sensors_level(r, v);
  collide_interior_hrr(r, v);
  if (l >= 1) {
    if (first_substep) parent_strain(r, l - 1);
    collide_boundary_hrr(r, l, wt);
  }
  v->nsteps++;
}

static void advance(orc_run* r, int l, const double* wt) {
  level_t* v = &r->lev[l];
  stream_level(r, v);
  if (l >= 1) rebuild_boundary(r, l, wt);
  if (l + 1 < r->nlev) {
    capture_history(r, l);
    double wA[3], wB[3] = {0.0, 0.0, 1.0};
    time_weights(v->nsteps == 0, wA);
    advance(r, l + 1, wA); /* asynchronous sub-step: t -> t+1/2 */
    advance(r, l + 1, wB); /* synchronous sub-step: t+1/2 -> t+1 */
    restrict_tn(r, l);
  }
  sensors_level(r, v);
  collide_level(r, v);
  v->nsteps++;
}

int orc_step(orc_run* r, int n) {
  for (int s = 0; s < n; ++s) {
    if (r->coll == 3)
      advance_hrr(r, 0, NULL, 0);
    else
      advance(r, 0, NULL);
  }
  return 0;
}

int orc_set_sigma(orc_run* r, double sigma) {
  if (!(sigma >= 0.0 && sigma <= 1.0)) return -1;
  r->sigma = sigma;
  return 0;
}

int orc_macros(const orc_run* r, int level, double* rho, double* u) {
  if (level < 0 || level >= r->nlev) return -1;
  const level_t* v = &r->lev[level];
  const int q = r->L.q;
#pragma omp parallel for schedule(static)
  for (long id = 0; id < v->N; ++id) {
    if (v->cls[id] == C_INACTIVE) {
      rho[id] = NAN;
      u[id] = u[v->N + id] = u[2 * v->N + id] = NAN;
      continue;
    }
    double rr, uu[3];
    moments(&r->L, v->fpost + id * q, &rr, uu);
    rho[id] = rr;
    u[id] = uu[0];
    u[v->N + id] = uu[1];
    u[2 * v->N + id] = uu[2];
  }
  return 0;
}

int orc_populations(const orc_run* r, int level, double* f) {
  if (level < 0 || level >= r->nlev) return -1;
  const level_t* v = &r->lev[level];
  const int q = r->L.q;
  for (long id = 0; id < v->N; ++id)
    for (int i = 0; i < q; ++i) f[(size_t)i * v->N + id] = v->fpost[id * q + i];
  return 0;
}
