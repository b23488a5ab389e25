// The loop of Sec. 3.8 (steps 2-9) over caller-supplied analyses: the
// normalised constraints of Eq. 3.21, the augmented-Lagrangian scalars of
// Eqs. 3.11-3.12 and the weights of Eq. 3.18, the return to the last feasible
// design with a halved volume step (steps 4 and 9), the target lowered once
// J has settled (steps 7-8), and the level-set cut (steps 5-6) delegated to
// the caller.  Host code only; afd_constrained_topology runs it on a mesh and
// afd_topology_run with the caller's callbacks.
#pragma once

#include <cmath>
#include <limits>

#include "afd.h"

namespace afd {

inline bool topo_active(const afd_topology_spec& s, int c) { return s.bound[c] > 0.0 && std::isfinite(s.bound[c]); }

// Upper bounds (compliance, stress) and lower bounds (eigenvalue, buckling).
inline double topo_g(int c, double value, double bound, double ref) {
  const double a = value / (bound * ref);
  return (c == AFD_CON_EIGEN || c == AFD_CON_BUCKLING) ? 1.0 - a : a - 1.0;
}

// Checks a spec; returns nullptr when valid, else the reason.
inline const char* topo_check(const afd_topology_spec& s) {
  bool any = false;
  for (int c = 0; c < AFD_CON_COUNT; ++c) {
    if (topo_active(s, c)) any = true;
    if (s.soft[c] && (c == AFD_CON_COMPLIANCE || c == AFD_CON_STRESS))
      return "only the eigenvalue and buckling constraints can be soft";
  }
  if (!any) return "no active constraint (every bound <= 0)";
  if (!(s.dv0 > 0.0 && s.dv0 < 1.0)) return "dv0 must be in (0, 1)";
  if (!(s.conv >= 0.0)) return "conv must be >= 0";
  if (s.max_fea < 1) return "max_fea must be >= 1";
  if (!(s.tol > 0.0)) return "tol must be > 0";
  if (topo_active(s, AFD_CON_STRESS) && !(s.p >= 1.0)) return "p must be >= 1";
  return nullptr;
}

template <typename Analyse, typename Save, typename Restore, typename Cut>
int topology_loop(const afd_topology_spec& s, Analyse&& analyse, Save&& save_feasible, Restore&& restore_feasible,
                  Cut&& cut, afd_topology_record* hist, int hist_cap, afd_topology_result* res) {
  const double nan = std::numeric_limits<double>::quiet_NaN();
  bool act[AFD_CON_COUNT], hard[AFD_CON_COUNT];
  afd_al_state al[AFD_CON_COUNT];
  for (int c = 0; c < AFD_CON_COUNT; ++c) {
    act[c] = topo_active(s, c);
    hard[c] = act[c] && !s.soft[c];
    afd_al_init(&al[c]);
  }
  const double dv_min = s.dv_min > 0.0 ? s.dv_min : 0.1 * s.dv0;
  double val[AFD_CON_COUNT], ref[AFD_CON_COUNT], g[AFD_CON_COUNT], w[AFD_CON_COUNT];
  for (int c = 0; c < AFD_CON_COUNT; ++c) val[c] = nan;
  int iters = 0;
  double rel = nan;
  int rc = analyse(0, val, &iters, &rel);
  if (rc != AFD_OK) return rc;
  int fea = 1;
  for (int c = 0; c < AFD_CON_COUNT; ++c) ref[c] = (act[c] || c == AFD_CON_COMPLIANCE) ? val[c] : nan;
  rc = save_feasible();
  if (rc != AFD_OK) return rc;
  double feasible_v = 1.0, v_design = 1.0, dv = s.dv0, v_target = 1.0 - s.dv0;
  bool have_prev = false;
  double J_prev = 0.0;
  int stop = AFD_STOP_MAX_FEA, n = 0;
  for (;;) {
    bool violated = false;
    for (int c = 0; c < AFD_CON_COUNT; ++c) {
      if (!act[c]) { g[c] = nan; continue; }
      g[c] = topo_g(c, val[c], s.bound[c], ref[c]);
      afd_al_update(&al[c], g[c]);
      if (hard[c] && g[c] > 0.0) violated = true;
    }
    // the record holds the state before this analysis' decision
    if (n < hist_cap && hist) {
      afd_topology_record& r = hist[n];
      r.fea = fea;
      r.v = v_design;
      r.target = v_target;
      r.dv = dv;
      for (int c = 0; c < AFD_CON_COUNT; ++c) {
        // J is analysed every time (it decides convergence) even when it is not constrained
        r.value[c] = (act[c] || c == AFD_CON_COMPLIANCE) ? val[c] : nan;
        r.g[c] = g[c];
        r.mu[c] = act[c] ? al[c].mu : nan;
        r.gamma[c] = act[c] ? al[c].gamma : nan;
      }
      r.violated = violated ? 1 : 0;
      r.iters = iters;
      r.rel_residual = rel;
    }
    ++n;
    if (fea >= s.max_fea) break;
    if (violated) {
      // steps 4 and 9: back to the last feasible design with half the step
      dv *= 0.5;
      if (dv < dv_min) {
        stop = AFD_STOP_DV_MIN;
        break;
      }
      rc = restore_feasible();
      if (rc != AFD_OK) return rc;
      v_design = feasible_v;
      v_target = feasible_v - dv;
      rc = analyse(1, val, &iters, &rel);
      if (rc != AFD_OK) return rc;
      ++fea;
      have_prev = false;
    } else {
      rc = save_feasible();
      if (rc != AFD_OK) return rc;
      feasible_v = v_design;
      // steps 7-8: J settled at this target -> the next target
      if (have_prev && std::fabs(val[AFD_CON_COMPLIANCE] - J_prev) <= s.conv * std::fabs(J_prev)) {
        if (v_target - dv < s.v_min) {
          stop = AFD_STOP_V_MIN;
          break;
        }
        v_target -= dv;
      }
      J_prev = val[AFD_CON_COMPLIANCE];
      have_prev = true;
    }
    for (int c = 0; c < AFD_CON_COUNT; ++c) w[c] = act[c] ? afd_al_weight(&al[c]) : 0.0;
    rc = cut(w, v_target);
    if (rc != AFD_OK) return rc;
    v_design = v_target;
    rc = analyse(1, val, &iters, &rel);
    if (rc != AFD_OK) return rc;
    ++fea;
  }
  if (res) {
    res->stop = stop;
    res->fea = fea;
    res->n_records = n;
    res->volume_fraction = feasible_v;
    for (int c = 0; c < AFD_CON_COUNT; ++c) res->reference[c] = ref[c];
  }
  return AFD_OK;
}

}  // namespace afd
