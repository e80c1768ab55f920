// host_common.h - host-side helpers shared by the single-run and the server
// entry points: argument checks, the gas-column tables, and the
// pass-independent part of the kernel parameters.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/karl.h"
#include "karl_device.cuh"

namespace karl {

// A named range on a profiler's timeline (NVTX): passes, cycles, field
// builds and server launches show up by name in Nsight; without a tool
// attached the calls do nothing.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

constexpr double HOST_Q_ENERGY = 16777216.0;    // 2^24 units per eV
constexpr double HOST_KB_EV = 8.617333262e-5;   // Boltzmann constant, eV/K

// Three-body clustering coefficients (k_ter / v, of order 1e-44 m^5) lie below
// the FP32 range.  Their table rows are kept multiplied by 2^128 and the n^2
// field by 2^-128: a power-of-two rescaling of both factors, exact in FP64,
// that leaves every product sigma n^2 unchanged.
constexpr double THREE_BODY_SCALE = 340282366920938463463374607431768211456.0;   // 2^128
constexpr double THREE_BODY_HALF_INV = 1.0 / 18446744073709551616.0;             // 2^-64

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

// Checks of the scattering-angle tables (no CUDA call): sets only on elastic
// channels, ordered energy ranges, non-negative pdfs with a positive integral
// in every bin.
inline bool angular_ok(const karl_xs* x) {
  const karl_angular* a = x->angular;
  if (!a) return true;
  if (a->n_sets < 1 || a->n_sets > KARL_MAX_CHANNELS || a->n_bins < 1 || a->n_bins > (1 << 16) ||
      a->n_mu < 2 || a->n_mu > 4096 || !a->set || !a->e_min_ev || !a->e_max_ev ||
      !a->threshold_ev || !a->pdf)
    return false;
  for (int k = 0; k < x->n_channels; ++k) {
    const int s = a->set[k];
    if (s < -1 || s >= a->n_sets || (s >= 0 && x->kind[k] != ELASTIC)) return false;
  }
  for (int s = 0; s < a->n_sets; ++s) {
    if (!(a->e_min_ev[s] > 0) || !(a->e_max_ev[s] > a->e_min_ev[s]) ||
        !host_finite(a->e_max_ev[s]) || !(a->threshold_ev[s] >= 0) ||
        !host_finite(a->threshold_ev[s]))
      return false;
    for (int b = 0; b < a->n_bins; ++b) {
      const double* p = a->pdf + ((size_t)s * a->n_bins + b) * a->n_mu;
      double sum = 0.0;
      for (int i = 0; i < a->n_mu; ++i) {
        if (!(p[i] >= 0) || !host_finite(p[i])) return false;
        sum += p[i];
      }
      if (!(sum > 0) || !host_finite(sum)) return false;
    }
  }
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
    if (kd < 0 || kd > CLUSTERING3 || si < 0 || si >= NSP || so < -1 || so >= NSP ||
        !(x->loss_ev[k] >= 0) || !host_finite(x->loss_ev[k]))
      return false;
    if ((kd == CLUSTERING || kd == CLUSTERING3 || kd == RECOMBINATION) && so < 0) return false;
    if (kd == CHARGE_EXCHANGE && si == SP_E) return false;
    if (x->target && (x->target[k] < 0 || x->target[k] > 1 ||
                      (x->target[k] == 1 && kd != ELASTIC && kd != IONIZATION)))
      return false;
    if (kd == RECOMBINATION && si != SP_E && so != SP_E) return false;
    if (kd == RECOMBINATION && si == SP_E && so == SP_E) return false;
    per_sp[si]++;
    if (field_kind(kd)) rec_sp[si]++;
    for (int i = 0; i < x->n_energy; ++i) {
      const double v = x->sigma_m2[(size_t)k * x->n_energy + i];
      if (!(v >= 0) || !host_finite(v)) return false;
      if (kd == CLUSTERING3 && !(v < 1e250)) return false;       // stays finite when scaled
    }
  }
  for (int s = 0; s < NSP; ++s)
    if (per_sp[s] > MAXSPCH || rec_sp[s] > 2) return false;
  return angular_ok(x);
}

// Gas column to each face, face positions (the last face is L exactly), the
// inverse density of each segment (0 without gas), and the inverse column on
// nq even steps (a search bracket for the flights).
struct ColumnTables {
  std::vector<double> col, faces, invn;
  std::vector<int> ginv;
  int nq = 0;
  double colmax = 0.0;
};

inline ColumnTables column_tables(const double* nseg, int nz, double length) {
  ColumnTables t;
  const double dz = length / nz;
  t.col.assign(nz + 1, 0.0);
  t.invn.assign(nz, 0.0);
  for (int j = 0; j < nz; ++j) {
    t.col[j + 1] = t.col[j] + nseg[j] * dz;
    t.invn[j] = nseg[j] > 0 ? 1.0 / nseg[j] : 0.0;
  }
  t.faces.resize(nz + 1);
  for (int k = 0; k < nz; ++k) t.faces[k] = (double)k * dz;
  t.faces[nz] = length;
  t.colmax = t.col[nz];
  t.nq = t.colmax > 0 ? std::min(8192, std::max(256, nz)) : 0;
  t.ginv.assign(t.nq + 1, 0);
  for (int q = 0, k = 0; q <= t.nq; ++q) {
    const double c = (double)q * t.colmax / t.nq;
    while (k < nz && t.col[k + 1] <= c) ++k;
    t.ginv[q] = k;
  }
  return t;
}

// Gas density squared per segment (times 2^-128) and its column to each face:
// the field of three-body clustering, whose rate per unit path is sigma n^2.
inline void square_column(const double* nseg, int nz, double length, std::vector<double>& n2,
                          std::vector<double>& col2) {
  const double dz = length / nz;
  n2.resize(nz);
  col2.assign(nz + 1, 0.0);
  for (int j = 0; j < nz; ++j) {
    const double h = nseg[j] * THREE_BODY_HALF_INV;
    n2[j] = h * h;
    col2[j + 1] = col2[j] + n2[j] * dz;
  }
}

inline bool has_kind(const karl_xs* x, int kind) {
  for (int k = 0; k < x->n_channels; ++k)
    if (x->kind[k] == kind) return true;
  return false;
}

// The physics model shared by every run of a context or server.
struct ModelInfo {
  int n_energy = 0;
  double e_min = 1, e_max = 2, eps_ion = 8;
  int nch = 0;
  int kind[MAXCH], sin[MAXCH], sout[MAXCH], target[MAXCH];
  double loss[MAXCH];
  // scattering-angle tables: set of each channel (-1 isotropic) and the sets'
  // energy ranges; the pdf values go to the device separately
  int ang[MAXCH];
  int ang_sets = 0, ang_nb = 0, ang_nmu = 0;
  double ang_lo[MAXCH], ang_hi[MAXCH], ang_thr[MAXCH];
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
    m.ang[k] = x->angular ? x->angular->set[k] : -1;
  }
  if (const karl_angular* a = x->angular) {
    m.ang_sets = a->n_sets;
    m.ang_nb = a->n_bins;
    m.ang_nmu = a->n_mu;
    for (int s = 0; s < a->n_sets; ++s) {
      m.ang_lo[s] = a->e_min_ev[s];
      m.ang_hi[s] = a->e_max_ev[s];
      m.ang_thr[s] = a->threshold_ev[s];
    }
  }
  return m;
}

// Device copies of the angle tables: the pdf rows and their cumulative
// integrals C(x_0) = 0, C(x_i+1) = C(x_i) + h (p_i + p_i+1) / 2 (exact for a
// pdf linear between the points), in FP64 and FP32.  Empty without tables.
inline void angular_tables(const karl_xs* x, std::vector<double>& pdf, std::vector<double>& cum,
                           std::vector<float>& pdff, std::vector<float>& cumf) {
  pdf.clear(); cum.clear(); pdff.clear(); cumf.clear();
  const karl_angular* a = x->angular;
  if (!a) return;
  const int n = a->n_mu;
  const size_t rows = (size_t)a->n_sets * a->n_bins;
  const double h = 2.0 / (double)(n - 1);
  pdf.assign(a->pdf, a->pdf + rows * n);
  cum.assign(rows * n, 0.0);
  for (size_t r = 0; r < rows; ++r) {
    const double* p = pdf.data() + r * n;
    double* c = cum.data() + r * n;
    for (int i = 0; i + 1 < n; ++i) c[i + 1] = c[i] + 0.5 * h * (p[i] + p[i + 1]);
  }
  pdff.assign(pdf.begin(), pdf.end());
  cumf.assign(cum.begin(), cum.end());
}

// Gas channels (rate sigma n(z)) that lead species s's selection order and
// are followed by field channels only: their count (0 with field channels
// only), or -1 when a gas channel follows a field channel (then every flight
// takes the per-channel path).
inline int leading_gas_channels(const ModelInfo& m, int s) {
  int n = 0;
  bool field_seen = false;
  for (int k = 0; k < m.nch; ++k) {
    if (m.sin[k] != s) continue;
    if (field_kind(m.kind[k])) field_seen = true;
    else if (field_seen) return -1;
    else ++n;
  }
  return n;
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
    P.ch[k].ang = m.ang[k];
  }
  if (m.ang_sets > 0) {
    P.ang_nb = m.ang_nb;
    P.ang_nmu = m.ang_nmu;
    P.ang_h = 2.0 / (double)(m.ang_nmu - 1);
    P.ang_inv_h = 0.5 * (double)(m.ang_nmu - 1);
    for (int s = 0; s < m.ang_sets; ++s) {
      P.ang_inv_lo[s] = 1.0 / m.ang_lo[s];
      P.ang_scale[s] = (double)m.ang_nb / std::log(m.ang_hi[s] / m.ang_lo[s]);
      P.ang_thr[s] = m.ang_thr[s];
    }
  }
  for (int s = 0; s < NSP; ++s) {
    int n = 0;
    for (int k = 0; k < m.nch; ++k) {
      if (m.sin[k] != s) continue;
      if (m.kind[k] == RECOMBINATION && pass != 2) continue;
      if (n < MAXSPCH) P.sc[s][n++] = (int8_t)k;
    }
    P.nsc[s] = n;
    P.ncg[s] = leading_gas_channels(m, s);
    P.cum_off[s] = s == 0 ? 0 : P.cum_off[s - 1] + std::max(P.ncg[s - 1], 0) * m.n_energy;
    P.mass[s] = g.species_mass_ev[s];
    P.inv_mass[s] = 1.0 / g.species_mass_ev[s];
    P.gam[s] = g.species_mass_ev[s] / g.target_mass_ev;
    P.gam2[s] = 2.0 * P.gam[s];
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

// Cumulative gas cross sections for the channel choice and the total rate.
// For species s, node interval i and its c-th leading gas channel, the sum
// over channels 0..c that are open across the whole interval (E_i above the
// channel's loss) of the node value and of the difference to the next node:
// sigma_0 + ... + sigma_c at energy E in the interval is value + t * slope,
// t the position of ln E in the interval.  An interval inside which exactly
// one channel opens is marked with that channel's slot (its own term is
// added above its threshold); one where two or more open is marked for the
// per-channel path.  The last row (index n_energy - 1, no interval above it)
// holds energies below the first node: there the tables are clamped to the
// first node and a channel is open at any energy when its loss is zero,
// closed when its loss is at or above the first node; a loss between the two
// sends the species to the per-channel path there.  Layout: species s from
// offset sum_{s' < s} max(ncg(s'), 0) * n_energy, then [row][channel] pairs
// (value, slope); marks [NSP][n_energy].
inline void gas_cum_tables(const karl_xs* x, const ModelInfo& m, std::vector<double>& cum,
                           std::vector<float>& cumf, std::vector<unsigned char>& mixed) {
  const int ne = x->n_energy;
  cum.clear();
  mixed.assign((size_t)NSP * ne, CUM_PER_CHANNEL);
  for (int s = 0; s < NSP; ++s) {
    const int ng = leading_gas_channels(m, s);
    if (ng < 0) continue;
    if (ng == 0) {                          // field channels only: nothing to add
      for (int i = 0; i < ne; ++i) mixed[(size_t)s * ne + i] = CUM_PLAIN;
      continue;
    }
    std::vector<int> ks;
    for (int k = 0; k < m.nch && (int)ks.size() < ng; ++k)
      if (m.sin[k] == s) ks.push_back(k);
    const size_t base = cum.size();
    cum.resize(base + (size_t)ne * ng * 2, 0.0);
    for (int i = 0; i + 1 < ne; ++i) {
      const double ei = m.e_min * std::pow(m.e_max / m.e_min, (double)i / (ne - 1));
      const double ej = m.e_min * std::pow(m.e_max / m.e_min, (double)(i + 1) / (ne - 1));
      int n_mix = 0, slot = -1;
      double a = 0.0, b = 0.0;
      for (int c = 0; c < ng; ++c) {
        const int k = ks[c];
        const double loss = m.loss[k];
        // margins of 1e-5 cover the rounding of ln E into the interval index
        // (FP32 in the precision form); an interval is 0.5 % of E wide
        const bool open = ei > loss * (1.0 + 1e-5) + 1e-300;
        const bool closed = ej * (1.0 + 1e-5) <= loss;
        if (!open && !closed) { ++n_mix; slot = c; }
        if (open) {
          const double v = x->sigma_m2[(size_t)k * ne + i];
          const double vn = x->sigma_m2[(size_t)k * ne + i + 1];
          a += v;
          b += vn - v;
        }
        cum[base + ((size_t)i * ng + c) * 2] = a;
        cum[base + ((size_t)i * ng + c) * 2 + 1] = b;
      }
      mixed[(size_t)s * ne + i] =
          n_mix == 0 ? CUM_PLAIN : (n_mix == 1 ? (unsigned char)slot : CUM_PER_CHANNEL);
    }
    // below the first node (clamped to it)
    bool uniform = true;
    double a = 0.0;
    for (int c = 0; c < ng; ++c) {
      const int k = ks[c];
      const double loss = m.loss[k];
      if (loss > 0.0 && loss < m.e_min) uniform = false;
      if (loss == 0.0) a += x->sigma_m2[(size_t)k * ne];
      cum[base + ((size_t)(ne - 1) * ng + c) * 2] = a;
      cum[base + ((size_t)(ne - 1) * ng + c) * 2 + 1] = 0.0;
    }
    mixed[(size_t)s * ne + ne - 1] = uniform ? CUM_PLAIN : CUM_PER_CHANNEL;
  }
  cumf.assign(cum.begin(), cum.end());
}

inline bool has_recombination(const ModelInfo& m) {
  for (int k = 0; k < m.nch; ++k)
    if (m.kind[k] == RECOMBINATION) return true;
  return false;
}

// [node][channel][2] copies of the cross sections for the transport kernels:
// each node's value and its difference to the next node (0 at the last), all
// channels of one node adjacent, so one 16-byte (8-byte in FP32) load gives
// both terms of the linear interpolation; three-body rows times 2^128.
inline void node_major_tables(const karl_xs* x, std::vector<double>& sig_t, std::vector<float>& sigf) {
  const int ne = x->n_energy, nc = x->n_channels;
  const size_t n = (size_t)nc * ne * 2;
  sig_t.assign(n, 0.0);
  sigf.assign(n, 0.0f);
  for (int k = 0; k < nc; ++k) {
    const double scale = x->kind[k] == CLUSTERING3 ? THREE_BODY_SCALE : 1.0;
    for (int i = 0; i < ne; ++i) {
      const double v = x->sigma_m2[(size_t)k * ne + i] * scale;
      const double vn = i + 1 < ne ? x->sigma_m2[(size_t)k * ne + i + 1] * scale : v;
      const size_t at = ((size_t)i * nc + k) * 2;
      sig_t[at] = v;
      sig_t[at + 1] = vn - v;
      const float f = (float)v, fn = (float)vn;
      sigf[at] = f;
      sigf[at + 1] = fn - f;
    }
  }
}

}  // namespace karl
