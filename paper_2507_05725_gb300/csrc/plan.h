// Host-side planning of one FTH-MS job: geometry of the overlapping arcs (Section 3.1), node
// counts, transfer meshes, chi, cross-evaluation targets, frequency and time grids (Section 5),
// and the offsets of every device array.  Everything here is O(nodes) or O(frequencies); all
// O(N^2) and larger work runs in the CUDA kernels.
#pragma once
#include <string>
#include <utility>
#include <vector>

#include "common.h"
#include "fthms.h"

namespace fthms {

struct Curve {
  std::vector<double> ax, bx, ay, by;
  void eval(double th, double& x, double& y, double& dx, double& dy) const;
};

struct ArcGeo {
  int curve;
  double ta, tb, tc, half;
  int prev = -1, next = -1;  // cyclic neighbours on the same curve (-1: open-arc obstacle)
  double length = 0.0;
};

struct Plan {
  std::vector<Curve> curves;
  std::vector<ArcGeo> arcs;
  fthms_signal sig{};
  std::vector<double> sig_f;  // samples of a sampled signal (copied from the caller)
  fthms_options opt{};
  std::vector<double> obs;  // 2 * n_obs
  int P = 0, L = 0, M = 0, Q = 0, K = 0, NT = 0, n_obs = 0, n_tout = 0;
  int lb = 1, le = 1;       // this rank's solved frequencies l in [lb, le) (all of 1..L-1 unpartitioned)
  int ranks = 1;            // frequency partition of the job (1 = none)
  bool own(int l) const { return l >= lb && l < le; }
  double h = 0, dt = 0, t0 = 0, H = 0, period = 0;
  std::vector<double> s_q, c_q;
  std::vector<int> nlo;
  std::vector<int> Ntab;  // [P][L] (column 0 unused)
  std::vector<int> Nmax;  // [P]

  std::vector<Panel> panels;
  std::vector<double> node_t, node_x, node_y, node_sp;
  std::vector<int> panel_index;  // [P][max N + 1] -> panel id or -1
  int maxN = 0;

  std::vector<SysDesc> sys;  // s = j*(L-1) + (l-1); systems of other ranks' frequencies have offsets -1
  std::vector<int> sys_order;  // systems by decreasing N: launch order of the per-system kernels
  int n_lu_big = 0;            // the first n_lu_big systems of sys_order take the tensor-core LU
  long long mat_total = 0, vec_total = 0, piv_total = 0;

  std::vector<int> rlogN;               // distinct N values
  std::vector<long long> rlog_off_N;    // offset per distinct N (same order)
  long long rlog_total = 0;

  std::vector<int> tpanel;              // transfer-mesh panel of arc k
  std::vector<long long> tr_off;        // offset of arc k's transfer nodes in chi / act arrays
  std::vector<double> chi;              // chi_k at transfer nodes, concatenated
  long long tr_total = 0;               // sum_k Nmax_k
  std::vector<int> act_off, act_idx;    // chi > 0 transfer nodes per arc (indices into the mesh)
  std::vector<int> act_arc;             // arc of each active node (global active list)

  std::vector<PairDesc> pairs;
  std::vector<CrossTgt> tgts;
  std::vector<long long> e_off;         // [pairs][L]
  long long e_total = 0;
  std::vector<CrossGrp> grps;
  std::vector<CrossBlk> blks;
  std::vector<ApplySlice> slices;       // row slices of the groups (mixed-form cross apply)
  std::vector<ResidChunk> rchunks;      // 32-row chunks of the systems, largest first (mixed-form residuals)
  std::vector<long long> grp_res_off;    // first row of each group in the per-row result buffer
  long long res_total = 0;               // rows over all groups
  int slice_ph_cap = 0;                  // max over slices of the summed N of the blocks it overlaps
  std::vector<CrossOtf> otf;            // cross_mode 1: on-the-fly tasks
  std::vector<long long> wn_off;         // per assembly task: offset of its near weights (nrows x N), or -1
  long long wn_total = 0;
  std::vector<long long> otf_res_off;    // [pairs][L]: first row of pair (k, j) in group (k, l)'s result rows
  std::vector<CrossAsm> asms;
  std::vector<SelfTile> self_tiles;

  std::vector<std::pair<int, int>> restr_pairs;  // (N, Nmax)
  std::vector<long long> restr_off;              // doubles offset per pair
  std::vector<long long> restr_of_sys;           // per system: table offset or -1 (identity)
  long long restr_total = 0;

  std::vector<double> win;   // [Q][NT]
  std::vector<double> wl;    // [L]
  std::vector<double> tout;  // [n_tout]

  long long spec_total = 0;  // sum_k Nmax_k * Q * L complex (transfer-node spectra)
  double hankel_self = 0, hankel_cross = 0;
  size_t device_bytes = 0;
};

// Returns FTHMS_OK or a status with a message in err.
int build_plan(const fthms_curve* curves, int ncurves, const fthms_arc* arcs, int narcs,
               const fthms_signal* sig, const fthms_options* opt, Plan& plan, std::string& err);

// The five launch choices (fthms_options.shapes, fthms_set_shapes) are among their candidates.
bool shapes_valid(const int* shapes, bool mixed);

// Offsets of the device arrays for a plan (bytes are accumulated into plan.device_bytes).
size_t plan_device_bytes(const Plan& p);

// First-kind nodes of one arc: t_i = cos((2i+1) pi/(2N)), x(t_i), y(t_i), |x'(t_i)|.
void arc_nodes(const Curve& c, double theta_a, double theta_b, int N, std::vector<double>& t,
               std::vector<double>& x, std::vector<double>& y, std::vector<double>& sp);

}  // namespace fthms
