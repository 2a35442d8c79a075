// Plain descriptors passed by value from the host scheduler to the kernels.
// They describe where a level's populations live and which nodes take part
// in each interface operation of the cell-vertex coupling (Sec. 4.3).
#pragma once
#include <cstdint>

namespace mlbm {

// One level's population storage: `batch` runs, each a set of q planes
// (structure of arrays), x fastest.  Node (x, y, z) has index
// e = off + (z * SY + y) * SX + x within a plane; plane i of run r holds it
// at element (r / es) * run_stride + (r % es) + i * plane + es * e.  es = 1:
// runs one after another.  es = 2 (binary16 storage with two or more runs):
// runs 2p and 2p+1 interleaved element by element, so one 4-byte access
// moves a node's population of both runs (plane and run_stride then count
// the interleaved elements).  Bounded axes carry a
// one-node ghost skin (x = -1 and x = n[0] on bounded x; y and z likewise);
// periodic axes wrap.  Rows are padded to a multiple of 32 elements so that
// node x = 0 of every row is 128-byte aligned for binary32 storage.
struct LevelView {
  void* f;
  long long plane;       // elements between consecutive planes of a run
  long long run_stride;  // q * plane: elements between runs (run pairs if es = 2)
  long long off;
  int n[3];
  int per[3];
  int SX, SY;
  int batch;
  // Parent nodes strictly inside the child's restriction ring are not
  // updated (inactive); empty when the level has no child.
  int has_ina;
  int ina_lo[3], ina_hi[3];
  // The restriction ring and what it encloses (TN nodes = this box minus
  // the inactive one); empty when the level has no child.
  int has_tn;
  int tn_lo[3], tn_hi[3];
  // Hybrid collision: TN nodes are collided by the restriction and, on a
  // refined level, the outer node layer (bounded axes) in its own kernel,
  // after the parent's strain rate at t+1 exists.
  short hrr;
  // element stride of consecutive nodes (1 or 2).  (hrr and es share one
  // 4-byte word: the view stays 128 bytes, the size the level update was
  // tuned with -- at 136 bytes its odd-parity instance ran 14 % more
  // instructions.)
  short es;
};
static_assert(sizeof(LevelView) == 128, "LevelView is kept at 128 bytes");

// Non-hydrodynamic mode sensor state of one level (Sec. 7), laid out like
// the population planes: div[run * plane + e], curl[(run * nc + c) * plane
// + e] (nc = 1 in 2D, 3 in 3D), gn, flag[run * plane + e] (bit 0 spuriousAc,
// bit 1 spuriousS, bit 2 spuriousG).  eps: magnitude floor of the sign
// tests; g2: squared threshold of |f1G|.
struct SensorState {
  float* div;
  float* curl;
  float* gn;  // |f1G|, gn[run * plane + e]
  unsigned char* flag;
  int nc;
  float eps, g2;
};

// Reference state of the shifted storage: level arrays hold
// g_i = f_i - f0_i(rho0, U) (U = 0: the rest-state shift f_i - w_i rho0).
struct RefState {
  double rho0;
  double U[3];
};

// Analytic initial state evaluated on the device (kinds as in mlbm.h).
struct ICDesc {
  int kind;  // 0 uniform, 1 vortex (about z), 2 Gaussian pulse
  double u0[3], center[3], radius, amplitude, eps, drho;
};

// Node positions of a level in level-0 units: origin + h * index, wrapped
// into the periodic level-0 domain of size dom.
struct Placement {
  double origin[3], h;
  int dom[3];
};

// Region of level-0 nodes the noise diagnostic skips: nodes within `margin`
// cells of the child box (box-relative coordinates on bounded axes).
struct NoiseRegion {
  int boxed[3], lo[3], E[3], n[3], margin;
};

constexpr int kMaxFaces = 6;

// Threads per block of the FP64 diagnostic reduction.
constexpr int kDiagThreads = 256;

// Parent-level history of (drho, du_x, du_y, du_z, f1_0 .. f1_{q-1}) on the
// surface of a child box, extended by one parent cell past its edges, in
// three time slots (t-1, t, t+1).  Face f (axis[f], side[f]) has ext[f][a]
// entries along axis a; local index i_a maps to parent coordinate
// base[f][a] + i_a (wrapped on periodic parent axes).
// Layout: hist[((run * 3 + slot) * nv + v) * K + k].
struct RingDesc {
  float* hist;
  long long K;
  int nv;
  int nf;
  int axis[kMaxFaces], side[kMaxFaces];
  long long start[kMaxFaces + 1];
  int ext[kMaxFaces][3];
  int base[kMaxFaces][3];
  int pn[3];      // parent node counts
  int pper[3];    // parent periodic axes
  int boxed[3];   // child axes bounded by the box
};

// Child-level c->f boundary nodes (TF and IE, the outer node layer of the
// child box), one entry per node: face f holds the nodes with x[axis] = 0
// (side 0) or n-1 (side 1) that lie on no earlier face; along axis a the
// face covers child coordinates lo[f][a] .. lo[f][a] + ext[f][a] - 1.
struct BndDesc {
  long long count;
  int nf;
  int axis[kMaxFaces], side[kMaxFaces];
  long long start[kMaxFaces + 1];
  int lo[kMaxFaces][3], ext[kMaxFaces][3];
};

// Face tiles of the child boundary for the tiled coarse -> fine rebuild:
// face f (axis[f], side[f]) spans the child nodes of the two tangent axes
// t1[f] < t2[f] (t2 = 2 with one node in 2D), cut into ntile1[f] x ntile2[f]
// tiles; tiles of face f are blocks tstart[f] .. tstart[f+1]-1.
struct InjDesc {
  int nf;
  int axis[kMaxFaces], side[kMaxFaces], t1[kMaxFaces], t2[kMaxFaces];
  int ntile1[kMaxFaces], ntile2[kMaxFaces];
  long long tstart[kMaxFaces + 1];
  int boxed[3];
};

// Tiles of TN nodes for the face-tiled restriction: face f's TN nodes form
// a rectangle along its tangent axes t1, t2; a tile covers up to TI x TJ of
// them (tiles of face f are numbered from tstart[f], t1 fastest).
struct RstDesc {
  int t1[kMaxFaces], t2[kMaxFaces];
  int ntile1[kMaxFaces];
  long long tstart[kMaxFaces + 1];
};

// Parent-level f->c nodes (TN, the parent nodes one parent cell inside the
// child box), one entry per node.  Face f covers box-relative coordinates
// rlo[f][a] .. rlo[f][a] + rext[f][a] - 1 along each axis (absolute parent
// coordinates on axes the box spans).
struct TnDesc {
  long long count;
  int nf;
  int axis[kMaxFaces], side[kMaxFaces];
  long long start[kMaxFaces + 1];
  int rlo[kMaxFaces][3], rext[kMaxFaces][3];
  int lo[3];      // child box lo (parent units)
  int boxed[3];
};

// Persistent fused step (kernels_fused.cuh): the recorded program, the
// launch arguments and the host-side description of the tables it reads.
constexpr int kFusedLevels = 4;
struct FusedTables;  // device tables (kernels_fused.cuh)

// One phase of a recorded coarse step.
struct Phase {
  int kind;     // 0 update, 1 capture, 2 rebuild, 3 restriction, 4 probe
  int level;    // update / rebuild / probe: that level; capture / restriction: the parent
  int par;      // update: its parity; capture: the parent's next update; rebuild: the
                // child's next update; restriction: the parent's next update; probe: last
  int cpar;     // restriction: the child's next update
  int slot[3];  // rebuild: history slots of t-1, t, t+1; capture: [0] the receiving slot
  float w[3];   // rebuild: temporal weights on those slots
  float resc;   // rebuild (eq. rescff) / restriction (eq. rescfc)
  float omega;  // update
  int nobar;    // 1: the next phase touches nothing this one does; no grid barrier between
};
constexpr int kFusedMaxPhases = 264;  // six coarse steps of four levels, cached in shared memory

struct FusedArgs {
  const FusedTables* tab;     // device
  const Phase* prog;          // device: the six programs back to back
  const int* prog_start;      // device [7]: program k is prog[prog_start[k] .. prog_start[k + 1])
  int first_key, nsteps;      // key of the first coarse step (its index mod 6), steps to take
  unsigned* bar;              // device [2]: arrival counter, generation
  int* err;                   // device: error word of this launch
  int* err_host;              // mapped host memory: the error word after the launch
  long long spin_limit;       // bounded waits
  int expect_extra;           // barrier expects this many blocks beyond the grid (0; tests > 0)
  int cluster;                // 1: the grid is one thread-block cluster (hardware barrier)
};

struct FusedHost {
  LevelView v[kFusedLevels];
  RingDesc ring[kFusedLevels];
  BndDesc bnd[kFusedLevels];
  TnDesc tn[kFusedLevels];
  RefState refd;
  int coll;
  int probe_n, probe_cap;
  const int* probe_ijk;
  double* probe_rec;
  unsigned long long* probe_counter;
};

}  // namespace mlbm
