// host_common.h - host-side helpers shared by the single-run and the server
// entry points: argument checks, the gas-column tables, and the
// pass-independent part of the kernel parameters.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/karl.h"
#include "karl_device.cuh"

namespace karl {

constexpr double HOST_Q_ENERGY = 16777216.0;    // 2^24 units per eV
constexpr double HOST_KB_EV = 8.617333262e-5;   // Boltzmann constant, eV/K

inline bool host_finite(double x) { return std::isfinite(x); }

// Geometry checks of karl_create (no CUDA call).
inline bool geometry_ok(const karl_geometry* g) {
  if (!g) return false;
  if (!(g->length_m > 0) || !host_finite(g->length_m) || g->n_zbins < 1 || g->n_zbins > (1 << 20) ||
      !g->n_seg_m3 || !(g->area_m2 > 0) || !(g->activity_bq > 0) || !(g->e_cut_ev >= 0) ||
      !(g->max_lifetime_s > 0) || !(g->gas_temperature_k >= 0) || g->n_tebins < 1 ||
      g->n_tebins > 4096 || g->n_spec_bins < 1 || g->n_spec_bins > (1 << 24) ||
      !(g->spec_bin_ev > 0) || !(g->target_mass_ev > 0) || !host_finite(g->gas_drift_mps) ||
      !(std::fabs(g->gas_drift_mps) < 1e7))
    return false;
  for (int s = 0; s < NSP; ++s)
    if (!(g->species_mass_ev[s] > 0)) return false;
  for (int j = 0; j < g->n_zbins; ++j)
    if (!(g->n_seg_m3[j] >= 0) || !host_finite(g->n_seg_m3[j])) return false;
  return true;
}

// Cross-section checks of karl_create (no CUDA call).
inline bool xs_ok(const karl_xs* x) {
  if (!x) return false;
  if (x->n_energy < 2 || !(x->e_min_ev > 0) || !(x->e_max_ev > x->e_min_ev) ||
      x->n_channels < 0 || x->n_channels > KARL_MAX_CHANNELS || !(x->ioniz_eps_ev > 0))
    return false;
  if (x->n_channels > 0 &&
      (!x->kind || !x->species_in || !x->species_out || !x->loss_ev || !x->sigma_m2))
    return false;
  int per_sp[NSP] = {0, 0, 0}, rec_sp[NSP] = {0, 0, 0};
  for (int k = 0; k < x->n_channels; ++k) {
    const int kd = x->kind[k], si = x->species_in[k], so = x->species_out[k];
    if (kd < 0 || kd > RECOMBINATION || si < 0 || si >= NSP || so < -1 || so >= NSP ||
        !(x->loss_ev[k] >= 0) || !host_finite(x->loss_ev[k]))
      return false;
    if ((kd == CLUSTERING || kd == RECOMBINATION) && so < 0) return false;
    if (x->target && (x->target[k] < 0 || x->target[k] > 1 || (x->target[k] == 1 && kd != ELASTIC)))
      return false;
    if (kd == RECOMBINATION && si != SP_E && so != SP_E) return false;
    if (kd == RECOMBINATION && si == SP_E && so == SP_E) return false;
    per_sp[si]++;
    if (kd == RECOMBINATION) rec_sp[si]++;
    for (int i = 0; i < x->n_energy; ++i) {
      const double v = x->sigma_m2[(size_t)k * x->n_energy + i];
      if (!(v >= 0) || !host_finite(v)) return false;
    }
  }
  for (int s = 0; s < NSP; ++s)
    if (per_sp[s] > MAXSPCH || rec_sp[s] > 2) return false;
  return true;
}

// Gas column to each face, face positions (the last face is L exactly), and
// the inverse column on nq even steps (a search bracket for the flights).
struct ColumnTables {
  std::vector<double> col, faces;
  std::vector<int> ginv;
  int nq = 0;
  double colmax = 0.0;
};

inline ColumnTables column_tables(const double* nseg, int nz, double length) {
  ColumnTables t;
  const double dz = length / nz;
  t.col.assign(nz + 1, 0.0);
  for (int j = 0; j < nz; ++j) t.col[j + 1] = t.col[j] + nseg[j] * dz;
  t.faces.resize(nz + 1);
  for (int k = 0; k < nz; ++k) t.faces[k] = (double)k * dz;
  t.faces[nz] = length;
  t.colmax = t.col[nz];
  t.nq = t.colmax > 0 ? std::min(8192, std::max(1024, 2 * nz)) : 0;
  t.ginv.assign(t.nq + 1, 0);
  for (int q = 0, k = 0; q <= t.nq; ++q) {
    const double c = (double)q * t.colmax / t.nq;
    while (k < nz && t.col[k + 1] <= c) ++k;
    t.ginv[q] = k;
  }
  return t;
}

// The physics model shared by every run of a context or server.
struct ModelInfo {
  int n_energy = 0;
  double e_min = 1, e_max = 2, eps_ion = 8;
  int nch = 0;
  int kind[MAXCH], sin[MAXCH], sout[MAXCH], target[MAXCH];
  double loss[MAXCH];
};

inline ModelInfo model_info(const karl_xs* x) {
  ModelInfo m;
  m.n_energy = x->n_energy;
  m.e_min = x->e_min_ev;
  m.e_max = x->e_max_ev;
  m.eps_ion = x->ioniz_eps_ev;
  m.nch = x->n_channels;
  for (int k = 0; k < x->n_channels; ++k) {
    m.kind[k] = x->kind[k];
    m.sin[k] = x->species_in[k];
    m.sout[k] = x->species_out[k];
    m.target[k] = x->target ? x->target[k] : 0;
    m.loss[k] = x->loss_ev[k];
  }
  return m;
}

// Everything of Params that does not depend on device buffers.
inline void fill_params(Params& P, const karl_geometry& g, const ModelInfo& m, int pass,
                        unsigned long long seed, int nq, double colmax) {
  std::memset(&P, 0, sizeof P);
  P.nz = g.n_zbins;
  P.L = g.length_m;
  P.dz = g.length_m / g.n_zbins;
  P.nq = nq;
  P.nq_over_colmax = colmax > 0 ? (double)nq / colmax : 0.0;
  P.nq_over_colmax_f = (float)P.nq_over_colmax;
  P.n_energy = m.n_energy;
  P.e_min = m.e_min;
  P.inv_e_min = 1.0 / m.e_min;
  P.log_ratio_h = std::log(m.e_max / m.e_min) / (double)(m.n_energy - 1);
  P.inv_h = 1.0 / P.log_ratio_h;
  P.nch = m.nch;
  for (int k = 0; k < m.nch; ++k) {
    P.ch[k].kind = m.kind[k];
    P.ch[k].sin = m.sin[k];
    P.ch[k].sout = m.sout[k];
    P.ch[k].target = m.target[k];
    P.ch[k].loss_q = (long long)std::floor(m.loss[k] * HOST_Q_ENERGY);
    P.ch[k].thr_q = (long long)std::floor(m.loss[k] * HOST_Q_ENERGY);
    P.ch[k].loss_ev = m.loss[k];
  }
  for (int s = 0; s < NSP; ++s) {
    int n = 0;
    for (int k = 0; k < m.nch; ++k) {
      if (m.sin[k] != s) continue;
      if (m.kind[k] == RECOMBINATION && pass != 2) continue;
      if (n < MAXSPCH) P.sc[s][n++] = (int8_t)k;
    }
    P.nsc[s] = n;
    P.mass[s] = g.species_mass_ev[s];
    P.inv_mass[s] = 1.0 / g.species_mass_ev[s];
    P.gam[s] = g.species_mass_ev[s] / g.target_mass_ev;
    P.inv_1pg2[s] = 1.0 / ((1.0 + P.gam[s]) * (1.0 + P.gam[s]));
  }
  P.target_mass = g.target_mass_ev;
  P.eps_ion = m.eps_ion;
  P.inv_eps_ion = 1.0 / m.eps_ion;
  P.kT = HOST_KB_EV * g.gas_temperature_k;
  P.drift_c = g.gas_drift_mps / 299792458.0;
  P.target_a = std::sqrt(P.kT / g.target_mass_ev);
  P.ecut_q = (long long)std::floor(g.e_cut_ev * HOST_Q_ENERGY);
  P.max_coll = g.max_collisions;
  P.max_life = g.max_lifetime_s;
  P.track_time = std::isfinite(g.max_lifetime_s) ? 1 : 0;
  P.ntb = g.n_tebins;
  P.tb_scale = g.n_tebins / std::log(m.e_max / m.e_min);
  P.nspec = g.n_spec_bins;
  P.spec_bin_q = (long long)std::llround(g.spec_bin_ev * HOST_Q_ENERGY);
  P.seed = seed;
  P.pass = pass;
}

inline bool has_recombination(const ModelInfo& m) {
  for (int k = 0; k < m.nch; ++k)
    if (m.kind[k] == RECOMBINATION) return true;
  return false;
}

// [node][channel] copies of the cross sections (all channels of one node in
// adjacent words) for the transport kernels.
inline void node_major_tables(const karl_xs* x, std::vector<double>& sig_t, std::vector<float>& sigf) {
  const size_t n = (size_t)x->n_channels * x->n_energy;
  sig_t.assign(n, 0.0);
  sigf.assign(n, 0.0f);
  for (int k = 0; k < x->n_channels; ++k)
    for (int i = 0; i < x->n_energy; ++i) {
      const double v = x->sigma_m2[(size_t)k * x->n_energy + i];
      sig_t[(size_t)i * x->n_channels + k] = v;
      sigf[(size_t)i * x->n_channels + k] = (float)v;
    }
}

}  // namespace karl
