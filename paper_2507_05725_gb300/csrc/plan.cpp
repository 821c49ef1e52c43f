// Host planning of an FTH-MS job (see plan.h).
#include "plan.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <map>
#include <thread>

namespace fthms {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoPi = 6.28318530717958647692;

double wrap_pi(double a) {
  double r = std::fmod(a + kPi, kTwoPi);
  if (r < 0) r += kTwoPi;
  r -= kPi;
  if (r <= -kPi) r += kTwoPi;
  return r;
}

// Smooth cut-off of eq. eta (Section 3.1).
double eta(double t, double t0, double t1) {
  t = std::fabs(t);
  if (t <= t0) return 1.0;
  if (t >= t1) return 0.0;
  double s = (t - t0) / (t1 - t0);
  return std::exp(2.0 * std::exp(-1.0 / s) / (s - 1.0));
}

// Time window sqcap of Section 5 (support [-H, H], equal to 1 on [-H/2, H/2]).
double window(double s, double H) {
  if (std::fabs(s) >= H) return 0.0;
  if (s >= -H / 2.0) return eta(s / H, 0.5, 1.0);
  return 1.0 - eta(s / H + 1.5, 0.5, 1.0);
}

// Clenshaw-Curtis rule on [-1, 1] with n+1 points (n even).
void clenshaw_curtis(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n + 1);
  w.resize(n + 1);
  for (int k = 0; k <= n; ++k) {
    double th = kPi * k / n;
    x[k] = std::cos(th);
    double s = 0.0;
    for (int j = 1; j <= n / 2; ++j) {
      double b = (2 * j == n) ? 1.0 : 2.0;
      s += b / (4.0 * j * j - 1.0) * std::cos(2.0 * j * th);
    }
    double c = (k == 0 || k == n) ? 1.0 : 2.0;
    w[k] = c / n * (1.0 - s);
  }
}

}  // namespace

void Curve::eval(double th, double& x, double& y, double& dx, double& dy) const {
  x = y = dx = dy = 0.0;
  for (size_t k = 0; k < ax.size(); ++k) {
    double c = std::cos(k * th), s = std::sin(k * th);
    x += ax[k] * c + bx[k] * s;
    y += ay[k] * c + by[k] * s;
    dx += k * (-ax[k] * s + bx[k] * c);
    dy += k * (-ay[k] * s + by[k] * c);
  }
}

namespace {

void arc_point(const Plan& p, int j, double t, double& x, double& y, double& sp) {
  const ArcGeo& a = p.arcs[j];
  double dx, dy;
  p.curves[a.curve].eval(a.tc + a.half * t, x, y, dx, dy);
  sp = std::hypot(dx, dy) * a.half;
}

double chi_at(const Plan& p, int j, double t) {
  const ArcGeo& a = p.arcs[j];
  if (a.next < 0) return 1.0;
  const Curve& c = p.curves[a.curve];
  double x, y, sp;
  arc_point(p, j, t, x, y, sp);
  double th = a.tc + a.half * t;
  double dum1, dum2;
  const ArcGeo& nx = p.arcs[a.next];
  const ArcGeo& pv = p.arcs[a.prev];
  // Right overlap Gamma_j cap Gamma_next: theta in [next.theta_a, theta_b].
  double dr = wrap_pi(th - nx.ta), span_r = wrap_pi(a.tb - nx.ta);
  if (t > 0 && dr >= 0.0 && dr <= span_r) {
    double ex, ey, fx, fy;
    c.eval(a.tb, ex, ey, dum1, dum2);
    c.eval(nx.ta, fx, fy, dum1, dum2);
    double A = std::hypot(fx - ex, fy - ey);
    double d = std::hypot(x - ex, y - ey);
    return eta(A - d, A / 3.0, 2.0 * A / 3.0);
  }
  // Left overlap Gamma_prev cap Gamma_j: theta in [theta_a, prev.theta_b].
  double dl = wrap_pi(pv.tb - th), span_l = wrap_pi(pv.tb - a.ta);
  if (t < 0 && dl >= 0.0 && dl <= span_l) {
    double ex, ey, fx, fy;
    c.eval(pv.tb, ex, ey, dum1, dum2);
    c.eval(a.ta, fx, fy, dum1, dum2);
    double A = std::hypot(fx - ex, fy - ey);
    double d = std::hypot(x - ex, y - ey);
    return 1.0 - eta(A - d, A / 3.0, 2.0 * A / 3.0);
  }
  return 1.0;
}

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }


}  // namespace

bool shapes_valid(const int* sh, bool mixed) {
  auto one_of = [](int v, std::initializer_list<int> ok) {
    if (v == 0) return true;
    for (int o : ok)
      if (v == o) return true;
    return false;
  };
  return one_of(sh[0], {1, 2, 4}) && one_of(sh[1], {64, 128, 256}) && one_of(sh[2], {128, 256, 512}) &&
         one_of(sh[3], {64, 128, 256}) && (mixed ? one_of(sh[4], {256, 384, 512, kLuBigMin}) : sh[4] == 0);
}

int build_plan(const fthms_curve* curves, int ncurves, const fthms_arc* arcs, int narcs,
               const fthms_signal* sig, const fthms_options* opt, Plan& p, std::string& err) {
  char buf[256];
  if (!curves || ncurves <= 0 || !arcs || narcs <= 0 || !sig || !opt) {
    err = "null or empty geometry/signal/options";
    return FTHMS_EINVAL;
  }
  p.opt = *opt;
  p.sig = *sig;
  if (opt->cross_mode != 0 && opt->cross_mode != 1) {
    err = "cross_mode must be 0 (stored cross rows) or 1 (evaluated every step)";
    return FTHMS_EINVAL;
  }
  if (opt->precision < 0 || opt->precision > 2) {
    err = "precision must be 0 (FP64), 1 (FP32 factors with double-float refinement and cross apply) or 2 (the "
          "same with FP64 small-argument Hankel series, refinement residuals and FFT butterflies)";
    return FTHMS_ENOTIMPL;
  }
  if (!(opt->refine_tol >= 0.0) || opt->refine_max < 0 || opt->refine_max > 16 ||
      (opt->refine_fallback != 0 && opt->refine_fallback != 1)) {
    err = "refine_tol must be >= 0, refine_max in [0, 16] and refine_fallback 0 or 1";
    return FTHMS_EINVAL;
  }
  if (!shapes_valid(opt->shapes, opt->precision >= 1)) {
    err = "shapes: a choice outside its candidates (solve warps {1, 2, 4}, assembly threads {64, 128, 256}, "
          "time threads {128, 256, 512}, restriction threads {64, 128, 256}, LU {256, 384, 512, 801} in the mixed "
          "forms and 0 in FP64; 0 = default)";
    return FTHMS_EINVAL;
  }
  if (p.opt.refine_tol == 0.0) p.opt.refine_tol = 1e-12;
  if (p.opt.refine_max == 0) p.opt.refine_max = 3;
  if (opt->L < 3 || !(opt->W > 0) || opt->M < 1 || opt->Q < 1 || !(opt->H > 0) ||
      !is_pow2(opt->n_period) || opt->n_period < 16 || opt->n_period > 16384 || opt->n_obs < 0 ||
      opt->n_tout < 0 || (opt->n_obs > 0 && !opt->obs_xy)) {
    err = "invalid options (need L >= 3, W > 0, M >= 1, Q >= 1, H > 0, n_period a power of two in [16, 16384])";
    return FTHMS_EINVAL;
  }
  if (opt->Q > 4) {
    err = "at most 4 time windows per job";
    return FTHMS_EINVAL;
  }
  if (opt->N_fixed <= 0 && (opt->N_min < 4 || !(opt->N_ppw >= 0))) {
    err = "node rule needs N_fixed > 0 or N_min >= 4";
    return FTHMS_EINVAL;
  }
  if (sig->kind != 0 && sig->kind != 1) {
    err = "signal kind must be 0 (point source) or 1 (plane wave)";
    return FTHMS_EINVAL;
  }
  if (sig->n_t == 0) {
    if (!(sig->width > 0)) {
      err = "signal width must be positive";
      return FTHMS_EINVAL;
    }
  } else {
    if (sig->n_t < 8 || sig->n_t > (1 << 24) || !sig->f || !(sig->dt > 0) || !std::isfinite(sig->t0) ||
        !(sig->band > 0) || !std::isfinite(sig->band)) {
      err = "sampled signal needs n_t in [8, 2^24], samples, dt > 0, a finite t0 and band > 0";
      return FTHMS_EINVAL;
    }
    p.sig_f.assign(sig->f, sig->f + sig->n_t);
    for (double v : p.sig_f)
      if (!std::isfinite(v)) {
        err = "sampled signal has a non-finite sample";
        return FTHMS_EINVAL;
      }
  }
  p.sig.f = nullptr;   // the samples live in p.sig_f (the caller's array may be freed)
  p.curves.resize(ncurves);
  for (int c = 0; c < ncurves; ++c) {
    const fthms_curve& cv = curves[c];
    if (cv.degree < 1 || !cv.ax || !cv.bx || !cv.ay || !cv.by) {
      err = "curve with degree < 1 or null coefficients";
      return FTHMS_EINVAL;
    }
    p.curves[c].ax.assign(cv.ax, cv.ax + cv.degree + 1);
    p.curves[c].bx.assign(cv.bx, cv.bx + cv.degree + 1);
    p.curves[c].ay.assign(cv.ay, cv.ay + cv.degree + 1);
    p.curves[c].by.assign(cv.by, cv.by + cv.degree + 1);
  }
  if (narcs > 64) {
    err = "at most 64 arcs per job";
    return FTHMS_EINVAL;
  }
  p.P = narcs;
  p.arcs.resize(narcs);
  for (int j = 0; j < narcs; ++j) {
    const fthms_arc& a = arcs[j];
    if (a.curve < 0 || a.curve >= ncurves || !(a.theta_b > a.theta_a) || a.theta_b - a.theta_a >= kTwoPi) {
      snprintf(buf, sizeof buf, "arc %d: bad curve index or parameter interval", j);
      err = buf;
      return FTHMS_EINVAL;
    }
    ArcGeo& g = p.arcs[j];
    g.curve = a.curve;
    g.ta = a.theta_a;
    g.tb = a.theta_b;
    g.tc = 0.5 * (a.theta_a + a.theta_b);
    g.half = 0.5 * (a.theta_b - a.theta_a);
  }
  // Cyclic neighbours per curve, ordered by centre angle (Section 3.1).
  for (int c = 0; c < ncurves; ++c) {
    std::vector<int> mine;
    for (int j = 0; j < narcs; ++j)
      if (p.arcs[j].curve == c) mine.push_back(j);
    if (mine.size() < 2) continue;
    std::sort(mine.begin(), mine.end(), [&](int a, int b) {
      double ca = std::fmod(p.arcs[a].tc, kTwoPi), cb = std::fmod(p.arcs[b].tc, kTwoPi);
      if (ca < 0) ca += kTwoPi;
      if (cb < 0) cb += kTwoPi;
      return ca < cb;
    });
    int n = (int)mine.size();
    for (int k = 0; k < n; ++k) {
      p.arcs[mine[k]].next = mine[(k + 1) % n];
      p.arcs[mine[k]].prev = mine[(k - 1 + n) % n];
    }
    // Each arc must overlap its neighbours, and the two overlaps must leave a truncated part.
    for (int k = 0; k < n; ++k) {
      const ArcGeo& a = p.arcs[mine[k]];
      const ArcGeo& nx = p.arcs[a.next];
      const ArcGeo& pv = p.arcs[a.prev];
      double span_r = wrap_pi(a.tb - nx.ta), span_l = wrap_pi(pv.tb - a.ta);
      double inner = 2.0 * a.half - span_r - span_l;
      if (!(span_r > 0) || !(span_l > 0) || !(inner > 0)) {
        snprintf(buf, sizeof buf, "arc %d: overlaps with its neighbours are empty or cover the whole arc", mine[k]);
        err = buf;
        return FTHMS_EINVAL;
      }
    }
  }
  {
    std::vector<double> xs, ws;
    clenshaw_curtis(256, xs, ws);
    for (int j = 0; j < narcs; ++j) {
      double s = 0.0, x, y, sp;
      for (size_t k = 0; k < xs.size(); ++k) {
        arc_point(p, j, xs[k], x, y, sp);
        s += ws[k] * sp;
      }
      p.arcs[j].length = s;
    }
  }

  // Frequency and time grids (Section 5 with the uniform-grid reading).
  p.L = opt->L;
  p.M = opt->M;
  p.Q = opt->Q;
  p.K = opt->n_period;
  p.H = opt->H;
  p.h = opt->W / (opt->L - 1);
  p.dt = kTwoPi / (p.h * p.K);
  p.t0 = -p.H;
  p.period = kTwoPi / p.h;
  if (p.period < 2.0 * p.H) {
    err = "window support 2H exceeds the period 2 pi/h of the frequency grid (increase L or reduce H)";
    return FTHMS_EINVAL;
  }
  p.s_q.resize(p.Q);
  p.c_q.resize(p.Q);
  p.nlo.resize(p.Q);
  for (int q = 0; q < p.Q; ++q) {
    p.s_q[q] = 1.5 * q * p.H;
    p.c_q[q] = p.h * (p.t0 - p.s_q[q]);
    p.nlo[q] = (int)std::ceil(p.s_q[q] / p.dt - 1e-9);
  }
  p.NT = (int)((p.s_q[p.Q - 1] + 2.0 * p.H) / p.dt) + 1;
  if (p.NT > 65536) {
    err = "internal time grid longer than 65536 samples";
    return FTHMS_EINVAL;
  }
  // The time kernels hold one period (n_period complex values) and the internal samples (NT doubles) of a
  // transfer node in shared memory.
  if ((size_t)p.K * 16 + (size_t)p.NT * 8 > (size_t)227 * 1024) {
    snprintf(buf, sizeof buf, "n_period (%d) and the internal time samples (%d) need %zu bytes of shared memory; "
             "at most 232448 (lower n_period, H or Q)", p.K, p.NT, (size_t)p.K * 16 + (size_t)p.NT * 8);
    err = buf;
    return FTHMS_EINVAL;
  }
  p.win.assign((size_t)p.Q * p.NT, 0.0);
  for (int q = 0; q < p.Q; ++q)
    for (int n = 0; n < p.NT; ++n) {
      double t = p.t0 + n * p.dt;
      p.win[(size_t)q * p.NT + n] = window(t - p.s_q[q], p.H);
    }
  // Frequency partition (Section 3: the per-frequency sub-problems of a step are independent): rank r of R
  // owns the solved frequencies l in [1 + r (L-1)/R, 1 + (r+1)(L-1)/R).
  if (opt->omega_ranks > 1) {
    if (opt->omega_rank < 0 || opt->omega_rank >= opt->omega_ranks || opt->omega_ranks > p.L - 1) {
      err = "omega partition needs 0 <= omega_rank < omega_ranks <= L - 1";
      return FTHMS_EINVAL;
    }
    p.ranks = opt->omega_ranks;
  } else if (opt->omega_rank != 0 || opt->omega_ranks < 0) {
    err = "omega_rank must be 0 without a frequency partition (omega_ranks <= 1)";
    return FTHMS_EINVAL;
  }
  {
    const long long ns = p.L - 1, R = p.ranks, r = p.ranks > 1 ? opt->omega_rank : 0;
    p.lb = 1 + (int)(r * ns / R);
    p.le = 1 + (int)((r + 1) * ns / R);
  }
  p.wl.assign(p.L, p.h);
  p.wl[0] = 0.0;
  p.wl[p.L - 1] = 0.5 * p.h;
  p.n_obs = opt->n_obs;
  p.obs.assign(opt->obs_xy, opt->obs_xy + 2 * (size_t)opt->n_obs);
  p.n_tout = opt->n_tout;
  p.tout.resize(p.n_tout);
  for (int i = 0; i < p.n_tout; ++i) p.tout[i] = opt->tout0 + opt->dtout * i;

  // Node counts N_j(omega_l).
  p.Ntab.assign((size_t)p.P * p.L, 0);
  p.Nmax.assign(p.P, 0);
  for (int j = 0; j < p.P; ++j) {
    for (int l = 1; l < p.L; ++l) {
      double omega = l * p.h;
      int N = opt->N_fixed > 0 ? opt->N_fixed
                               : std::max(opt->N_min, (int)std::ceil(opt->N_ppw * omega * p.arcs[j].length - 1e-9) + opt->N_off);
      const int nmax = opt->precision == 0 ? kLuSmallMax : kLuBigMax;
      if (N < 2 || N > nmax) {
        snprintf(buf, sizeof buf, "arc %d omega index %d: node count %d outside [2, %d] (%s)", j, l, N, nmax,
                 opt->precision == 0 ? "FP64: shared-memory panel of the LU; the mixed forms reach 2048"
                                     : "largest tensor-core LU");
        err = buf;
        return FTHMS_EINVAL;
      }
      p.Ntab[(size_t)j * p.L + l] = N;
      p.maxN = std::max(p.maxN, N);
    }
    p.Nmax[j] = p.Ntab[(size_t)j * p.L + p.L - 1];
    for (int l = 1; l < p.L; ++l)
      if (p.Ntab[(size_t)j * p.L + l] > p.Nmax[j]) {
        err = "node count must not decrease with frequency";
        return FTHMS_EINVAL;
      }
  }

  // Node panels (arc, N): t_i, x(t_i), |x'(t_i)|.  Panels met by the systems loop are only registered
  // there and filled afterwards on several threads (each panel independently, the same arithmetic).
  p.panel_index.assign((size_t)p.P * (p.maxN + 1), -1);
  long long noff = 0;
  std::vector<int> deferred;
  auto fill_panel = [&](int idx) {
    const Panel pn = p.panels[idx];
    for (int i = 0; i < pn.N; ++i) {
      const double t = std::cos((2.0 * i + 1.0) * kPi / (2.0 * pn.N));
      double x, y, sp;
      arc_point(p, pn.arc, t, x, y, sp);
      p.node_t[pn.off + i] = t;
      p.node_x[pn.off + i] = x;
      p.node_y[pn.off + i] = y;
      p.node_sp[pn.off + i] = sp;
    }
  };
  auto get_panel = [&](int j, int N, bool defer = false) {
    int& idx = p.panel_index[(size_t)j * (p.maxN + 1) + N];
    if (idx >= 0) return idx;
    idx = (int)p.panels.size();
    p.panels.push_back(Panel{j, N, noff});
    noff += N;
    p.node_t.resize(noff);
    p.node_x.resize(noff);
    p.node_y.resize(noff);
    p.node_sp.resize(noff);
    if (defer) deferred.push_back(idx);
    else fill_panel(idx);
    return idx;
  };

  // Systems, self tiles, distinct N for the log tables.
  std::map<int, long long> rlog_map;
  p.sys.resize((size_t)p.P * (p.L - 1));
  for (int j = 0; j < p.P; ++j)
    for (int l = 1; l < p.L; ++l) {
      int N = p.Ntab[(size_t)j * p.L + l];
      SysDesc& s = p.sys[(size_t)j * (p.L - 1) + (l - 1)];
      s.arc = j;
      s.l = l;
      s.N = N;
      s.kappa = l * p.h;
      if (!p.own(l)) {           // another rank's frequency: no storage here
        s.panel = -1;
        s.mat_off = s.vec_off = s.piv_off = s.rlog_off = -1;
        continue;
      }
      s.panel = get_panel(j, N, true);
      s.mat_off = p.mat_total;
      s.vec_off = p.vec_total;
      s.piv_off = p.piv_total;
      p.mat_total += (long long)N * N;
      p.vec_total += (long long)p.Q * N;
      p.piv_total += N;
      rlog_map[N] = 0;
      p.hankel_self += 0.5 * N * (N + 1.0);
    }
  {
    const int nthr = std::max(1, std::min(16, (int)std::thread::hardware_concurrency()));
    std::atomic<int> next{0};
    auto work = [&] {
      for (int k = next.fetch_add(1); k < (int)deferred.size(); k = next.fetch_add(1)) fill_panel(deferred[k]);
    };
    std::vector<std::thread> pool;
    if (nthr > 1 && deferred.size() >= 64) {
      try {
        for (int t = 1; t < nthr; ++t) pool.emplace_back(work);
      } catch (...) {   // no threads available: the calling thread fills the rest
      }
    }
    work();
    for (auto& t : pool) t.join();
  }
  // Self-assembly tiles over bands of consecutive frequencies with the same N.
  for (int j = 0; j < p.P; ++j) {
    int l = p.lb;
    while (l < p.le) {
      int N = p.Ntab[(size_t)j * p.L + l];
      int l1 = l;
      while (l1 + 1 < p.le && p.Ntab[(size_t)j * p.L + l1 + 1] == N && l1 + 1 - l < kSelfBand) ++l1;
      int nt = (N + kSelfTile - 1) / kSelfTile;
      int sidx = j * (p.L - 1) + (l - 1);
      for (int a = 0; a < nt; ++a)
        for (int b = a; b < nt; ++b) p.self_tiles.push_back(SelfTile{sidx, l1 - l + 1, a, b});
      l = l1 + 1;
    }
  }
  for (auto& kv : rlog_map) {
    kv.second = p.rlog_total;
    p.rlogN.push_back(kv.first);
    p.rlog_off_N.push_back(p.rlog_total);
    p.rlog_total += (long long)kv.first * kv.first;
  }
  for (auto& s : p.sys)
    if (p.own(s.l)) s.rlog_off = rlog_map[s.N];
  // Largest systems first, so that the last wave of the per-system kernels holds the small ones.
  for (size_t s = 0; s < p.sys.size(); ++s)
    if (p.own(p.sys[s].l)) p.sys_order.push_back((int)s);
  std::stable_sort(p.sys_order.begin(), p.sys_order.end(), [&](int a, int b) { return p.sys[a].N > p.sys[b].N; });
  // LU paths: the mixed forms factor systems of kLuBigMin nodes or more with tensor-core trailing updates
  // (a prefix of sys_order, which is sorted by decreasing N; fthms_autotune may move the threshold down).
  p.n_lu_big = 0;
  if (p.opt.precision >= 1)
    while (p.n_lu_big < (int)p.sys_order.size() && p.sys[p.sys_order[p.n_lu_big]].N >= kLuBigMin) ++p.n_lu_big;
  if (p.opt.precision >= 1)
    for (int s : p.sys_order)
      for (int r0 = 0; r0 < p.sys[s].N; r0 += 32) p.rchunks.push_back(ResidChunk{s, r0});

  // Transfer meshes, chi and the active (chi > 0) nodes.
  p.tpanel.resize(p.P);
  p.tr_off.resize(p.P);
  p.act_off.assign(p.P + 1, 0);
  for (int k = 0; k < p.P; ++k) {
    p.tpanel[k] = get_panel(k, p.Nmax[k]);
    p.tr_off[k] = p.tr_total;
    const Panel& pn = p.panels[p.tpanel[k]];
    p.act_off[k] = (int)p.act_idx.size();
    for (int x = 0; x < pn.N; ++x) {
      double c = chi_at(p, k, p.node_t[pn.off + x]);
      p.chi.push_back(c);
      if (c > 0.0) {
        p.act_idx.push_back(x);
        p.act_arc.push_back(k);
      }
    }
    p.tr_total += pn.N;
  }
  p.act_off[p.P] = (int)p.act_idx.size();
  p.spec_total = p.tr_total * (long long)p.Q * p.L;

  // Cross-evaluation pairs and targets (eq. vtilde masking; near rule for 1 < |t*| <= 3).
  for (int k = 0; k <= p.P; ++k) {
    for (int j = 0; j < p.P; ++j) {
      if (j == k) continue;
      PairDesc pd{k, j, (int)p.tgts.size(), 0};
      if (k == p.P) {
        for (int z = 0; z < p.n_obs; ++z) p.tgts.push_back(CrossTgt{p.obs[2 * z], p.obs[2 * z + 1], 0.0, 0, z});
      } else {
        const Panel& pn = p.panels[p.tpanel[k]];
        const ArcGeo& aj = p.arcs[j];
        const ArcGeo& ak = p.arcs[k];
        for (int a = p.act_off[k]; a < p.act_off[k + 1]; ++a) {
          int x = p.act_idx[a];
          double tx = p.node_t[pn.off + x];
          double X = p.node_x[pn.off + x], Y = p.node_y[pn.off + x];
          if (aj.curve == ak.curve) {
            double th = ak.tc + ak.half * tx;
            double ts = wrap_pi(th - aj.tc) / aj.half;
            if (std::fabs(ts) <= 1.0) continue;  // point of Gamma_j: dropped (eq. vtilde)
            int near = std::fabs(ts) <= 3.0 ? 1 : 0;
            p.tgts.push_back(CrossTgt{X, Y, near ? ts : 0.0, near, x});
          } else {
            p.tgts.push_back(CrossTgt{X, Y, 0.0, 0, x});
          }
        }
      }
      pd.nrows = (int)p.tgts.size() - pd.tgt_off;
      p.pairs.push_back(pd);
    }
  }
  int npairs = (int)p.pairs.size();
  p.e_off.assign((size_t)npairs * p.L, -1);
  for (int pi = 0; pi < npairs; ++pi) {
    const PairDesc& pd = p.pairs[pi];
    if (pd.nrows == 0) continue;
    for (int l = p.lb; l < p.le; ++l) {
      int N = p.Ntab[(size_t)pd.j * p.L + l];
      p.e_off[(size_t)pi * p.L + l] = p.e_total;
      p.e_total += (long long)pd.nrows * N;
    }
  }
  p.hankel_cross = (double)p.e_total;
  // Pairs with rows, per receiver, in pair order (the block order of every group).
  std::vector<std::vector<int>> pairs_of(p.P + 1);
  for (int pi = 0; pi < npairs; ++pi)
    if (p.pairs[pi].nrows > 0) pairs_of[p.pairs[pi].k].push_back(pi);
  p.blks.reserve((size_t)npairs * (p.le - p.lb));
  for (int l = p.lb; l < p.le; ++l)
    for (int k = 0; k <= p.P; ++k) {
      CrossGrp g{l, k, (int)p.blks.size(), 0};
      for (int pi : pairs_of[k]) {
        const PairDesc& pd = p.pairs[pi];
        int N = p.Ntab[(size_t)pd.j * p.L + l];
        CrossBlk b{pd.j, pd.j * (p.L - 1) + (l - 1), N, pd.nrows, pd.tgt_off, 0, p.e_off[(size_t)pi * p.L + l]};
        p.blks.push_back(b);
      }
      g.blk_end = (int)p.blks.size();
      if (g.blk_end > g.blk_begin) p.grps.push_back(g);
    }
  // Row slices for the mixed-form apply: kApplySlice consecutive rows of a group per CTA.
  p.grp_res_off.resize(p.grps.size());
  for (size_t gi = 0; gi < p.grps.size(); ++gi) {
    const CrossGrp& g = p.grps[gi];
    p.grp_res_off[gi] = p.res_total;
    int rows = 0;
    for (int b = g.blk_begin; b < g.blk_end; ++b) rows += p.blks[b].nrows;
    p.res_total += rows;
    // A slice ends early at a block boundary when the densities it stages (Q x summed N) would
    // exceed kSliceDensities complex values (196 KB of shared memory).
    const int kSliceDensities = 12288;
    int b = g.blk_begin, rb = 0;              // block containing row0 and its first row
    for (int row0 = 0; row0 < rows;) {
      while (row0 >= rb + p.blks[b].nrows) rb += p.blks[b++].nrows;
      int end = std::min(row0 + kApplySlice, rows);
      ApplySlice sl{(int)gi, row0, 0, b, b, rb};
      int nsum = p.blks[b].N, re = rb + p.blks[b].nrows;
      while (re < end) {
        if ((nsum + p.blks[sl.b1 + 1].N) * p.Q > kSliceDensities) {
          end = re;
          break;
        }
        ++sl.b1;
        nsum += p.blks[sl.b1].N;
        re += p.blks[sl.b1].nrows;
      }
      sl.nrows = end - row0;
      p.slice_ph_cap = std::max(p.slice_ph_cap, nsum);
      p.slices.push_back(sl);
      row0 = end;
    }
  }
  // Stored cross rows: the assembly keeps 4N + 2 kAsmRows N doubles and its band tables in shared memory.
  if (p.opt.cross_mode == 0 && (size_t)(20 * p.maxN + 512) * 8 > (size_t)227 * 1024) {
    snprintf(buf, sizeof buf, "stored cross rows (cross_mode 0) need N <= 1427 (largest N %d); use cross_mode 1", p.maxN);
    err = buf;
    return FTHMS_EINVAL;
  }
  const int kRowChunk = 8;
  // Assembly tasks: (pair, band of up to 64 equal-N frequencies, kRowChunk target rows); counted first so
  // that the list is filled without reallocation.
  auto band_end = [&](int j, int l) {
    const int N = p.Ntab[(size_t)j * p.L + l];
    int l1 = l;
    while (l1 + 1 < p.le && p.Ntab[(size_t)j * p.L + l1 + 1] == N && l1 + 1 - l < 64) ++l1;
    return l1;
  };
  size_t n_asm = 0;
  for (int pi = 0; pi < npairs; ++pi) {
    const PairDesc& pd = p.pairs[pi];
    if (pd.nrows == 0) continue;
    for (int l = p.lb; l < p.le; l = band_end(pd.j, l) + 1) n_asm += (pd.nrows + kRowChunk - 1) / kRowChunk;
  }
  p.asms.reserve(n_asm);
  for (int pi = 0; pi < npairs; ++pi) {
    const PairDesc& pd = p.pairs[pi];
    if (pd.nrows == 0) continue;
    int l = p.lb;
    while (l < p.le) {
      int N = p.Ntab[(size_t)pd.j * p.L + l];
      int l1 = band_end(pd.j, l);
      int panel = get_panel(pd.j, N);
      for (int r0 = 0; r0 < pd.nrows; r0 += kRowChunk)
        p.asms.push_back(CrossAsm{pi, l, l1, N, r0, std::min(kRowChunk, pd.nrows - r0), panel, 0});
      l = l1 + 1;
    }
  }
  if (p.opt.cross_mode == 1) {
    // Rows of pair (k, j) inside the per-row results of group (k, l), in the groups' block order.
    p.otf_res_off.assign((size_t)npairs * p.L, -1);
    for (size_t gi = 0; gi < p.grps.size(); ++gi) {
      const CrossGrp& g = p.grps[gi];
      long long r = p.grp_res_off[gi];
      for (int pi : pairs_of[g.k]) {
        p.otf_res_off[(size_t)pi * p.L + g.l] = r;
        r += p.pairs[pi].nrows;
      }
    }
    // Near weights once per job (they depend on the target and N only); tasks of at most
    // otf_band(Q) frequencies each.
    const int band = p.opt.precision >= 1 ? kOtfBandDf : otf_band(p.Q);
    p.wn_off.assign(p.asms.size(), -1);
    for (size_t a = 0; a < p.asms.size(); ++a) {
      const CrossAsm& t = p.asms[a];
      const PairDesc& pd = p.pairs[t.pair];
      bool near = false;
      for (int r = 0; r < t.nrows; ++r) near = near || p.tgts[pd.tgt_off + t.row0 + r].near;
      if (near) {
        p.wn_off[a] = p.wn_total;
        p.wn_total += (long long)t.nrows * t.N;
      }
      for (int l = t.l0; l <= t.l1; l += band) p.otf.push_back(CrossOtf{(int)a, l, std::min(l + band - 1, t.l1), 0});
    }
  }

  // Restriction tables (N, Nmax) for systems below their arc's transfer-mesh size.
  std::map<std::pair<int, int>, long long> rmap;
  p.restr_of_sys.assign(p.sys.size(), -1);
  for (size_t s = 0; s < p.sys.size(); ++s) {
    int N = p.sys[s].N, Nm = p.Nmax[p.sys[s].arc];
    if (N == Nm || !p.own(p.sys[s].l)) continue;
    auto key = std::make_pair(N, Nm);
    auto it = rmap.find(key);
    if (it == rmap.end()) {
      rmap[key] = p.restr_total;
      p.restr_pairs.push_back(key);
      p.restr_off.push_back(p.restr_total);
      p.restr_total += (long long)N * Nm;
      it = rmap.find(key);
    }
    p.restr_of_sys[s] = it->second;
  }
  p.device_bytes = plan_device_bytes(p);
  return FTHMS_OK;
}

void arc_nodes(const Curve& c, double theta_a, double theta_b, int N, std::vector<double>& t,
               std::vector<double>& x, std::vector<double>& y, std::vector<double>& sp) {
  const double tc = 0.5 * (theta_a + theta_b), half = 0.5 * (theta_b - theta_a);
  t.resize(N); x.resize(N); y.resize(N); sp.resize(N);
  for (int i = 0; i < N; ++i) {
    t[i] = std::cos((2.0 * i + 1.0) * kPi / (2.0 * N));
    double dx, dy;
    c.eval(tc + half * t[i], x[i], y[i], dx, dy);
    sp[i] = std::hypot(dx, dy) * half;
  }
}

size_t plan_device_bytes(const Plan& p) {
  size_t b = 0;
  b += (size_t)p.mat_total * 16;                 // A / LU
  if (p.opt.precision >= 1)                      // FP32 factors, residuals and corrections, refinement state
    b += (size_t)p.mat_total * 8 + (size_t)p.piv_total * 8 + (size_t)p.vec_total * (8 + 16 + 16 + 8) +
         p.sys.size() * (24 + 32) + (size_t)p.piv_total * 8 + p.rchunks.size() * sizeof(ResidChunk);
  b += p.sig_f.size() * 8;                       // samples of a sampled signal
  b += (size_t)p.piv_total * 4;                  // pivots
  b += (size_t)p.rlog_total * 8;                 // self log tables
  b += (size_t)p.vec_total * 16 * 3;             // G, phi (current), phi sum
  if (p.opt.keep_densities) b += (size_t)p.vec_total * 16 * p.M;
  b += (size_t)p.spec_total * 16 * 2;            // W and Gt on transfer meshes
  b += p.act_idx.size() * (size_t)p.NT * 8;      // m = 1 time samples at the active transfer nodes
  if (p.opt.cross_mode == 0) b += (size_t)p.e_total * 16;   // stored cross matrices
  b += (size_t)p.restr_total * (p.opt.precision >= 1 ? 16 : 8);
  b += (size_t)p.n_obs * p.Q * p.L * 16 + (size_t)p.n_obs * p.n_tout * 8;
  b += p.node_t.size() * 32 + p.tgts.size() * sizeof(CrossTgt) + p.blks.size() * sizeof(CrossBlk) +
       p.asms.size() * sizeof(CrossAsm) + p.self_tiles.size() * sizeof(SelfTile) + p.sys.size() * (sizeof(SysDesc) + sizeof(int)) + p.slices.size() * sizeof(ApplySlice) + p.grp_res_off.size() * 8;
  if (p.opt.precision >= 1 || p.opt.cross_mode == 1) b += (size_t)p.res_total * p.Q * 16;   // per-row cross sums
  if (p.opt.cross_mode == 1)
    b += (size_t)p.wn_total * 8 + p.otf.size() * sizeof(CrossOtf) + p.otf_res_off.size() * 8 + p.wn_off.size() * 8;
  b += p.win.size() * 8 + (size_t)p.Q * p.L * 32 + (size_t)p.K * (p.opt.precision >= 1 ? 16 : 8) + p.chi.size() * 8;
  return b;
}

}  // namespace fthms
