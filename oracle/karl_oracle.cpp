/*
 * karl_oracle.cpp - plain FP64 CPU oracle of the KARL transport step.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, by __graft_entry__.smoke()
 * and by bench.py's CPU-baseline leg, never by the product path.
 *
 * Each primary is followed event by event, with its products on a stack, the
 * way the paper's main cycle does (Sec. 2.1, Fig. 1): draw a free path from the
 * mean free path (Eqs. mean_free_path and distance_from_mfp), move, tally the
 * time spent per segment and the face crossings (Secs. 2.2-2.3), check the
 * terminator (Sec. 3.2), pick a channel with probability sigma_i n_i over the
 * total (Sec. 2.1), and perform it (Sec. 3.3).  Written for reading, not speed:
 * linear walks over segments, no tables beyond the inputs, FP64 throughout.
 *
 * Readings where the paper is silent (the same ones the GPU path follows):
 *  - gas density is piecewise constant per z segment; the magnetic field is
 *    uniform along z, so only z and the pitch cosine mu matter (drift mover,
 *    Sec. 3.1, exact for uniform B and no E field);
 *  - sigma(E): linear interpolation in ln E on the input nodes, zero for
 *    E <= loss of the channel, clamped to the end nodes outside the grid;
 *  - lab kinetic energy with the target at rest; relativistic speed;
 *  - elastic: isotropic in the centre-of-mass frame unless the channel has a
 *    scattering-angle table (Sec. 3.3 Elastic: the table's energy bin is
 *    chosen and cos chi drawn from its piecewise-linear pdf by inverting the
 *    cumulative integral; isotropic below the table's threshold energy, the
 *    composition the paper uses for electrons); the angle is the centre-of-
 *    mass polar angle, at the impact energy; for a channel marked as
 *    having a moving target (Sec. 3.3 Elastic: gas drift plus a Maxwell-
 *    Boltzmann velocity), nonrelativistic velocities, the impactor's gyrophase
 *    taken as 0 (the target distribution is symmetric about z), the relative
 *    velocity rotated in the centre-of-mass frame;
 *  - ionization: secondary energy W in [0, (E-I)/2] with pdf ~ 1/(1+(W/eps)^2),
 *    the fast electron is the incident one, binary-encounter polar angles,
 *    secondary azimuth = primary azimuth - pi (Sec. 3.3, Ionization); the ion
 *    gets a thermal target velocity (no recoil); for a channel with a moving
 *    target the target velocity is drawn as for elastic scattering and redrawn
 *    while the impact energy relative to it is not above I, the sharing and
 *    angles happen in the target's frame, the ion takes the target velocity,
 *    and the lab energy the gas gives or takes goes to the recoil ledger;
 *  - clustering: the product takes a thermal target's direction and the speed
 *    that keeps the target's kinetic energy with the product mass; three-body
 *    clustering (Sec. 3.3 Clustering, Eq. clustering_tertiary) has the rate
 *    per unit path sigma_k(E) n(z)^2, its table holding k_ter / v, so that the
 *    mean free path is v / (k_ter n^2) (Eq. clustering_test_tertiary_mfp);
 *  - charge exchange (Sec. 3.3 Charge exchange): the impactor takes the
 *    velocity of a target particle drawn as for a moving elastic target (gas
 *    drift plus a Maxwell-Boltzmann velocity with the relative-speed weight),
 *    keeps its species, and the change of kinetic energy goes to the gas;
 *  - recombination: the impactor is deleted, the partner's field logs one
 *    deletion in the segment (Sec. 3.3, Recombination);
 *  - two passes: pass 1 without recombination builds the target fields,
 *    pass 2 uses them frozen; or the paper's continuous update (Sec. 3.6):
 *    the primaries in consecutive cycles, each cycle with the fields of the
 *    cycles before it, deletions included (Eq. target_field_density), the
 *    first with fields of zero;
 *  - random numbers: Philox4x64-10 (Salmon et al., SC'11) keyed by
 *    (seed, primary id), counter (event index, lineage id, pass/domain, sub).
 */
#include "karl_oracle.h"

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

namespace {

const double C_LIGHT = 299792458.0;
const double KB_EV = 8.617333262e-5;
const double TWO_PI = 6.283185307179586476925286766559;
const double Q_ENERGY = 16777216.0;             /* 2^24 units per eV */
const double Q_TIME = 1125899906842624.0;       /* 2^50 units per s */

enum { ELASTIC = 0, IONIZATION = 1, EXCITATION = 2, CLUSTERING = 3, RECOMBINATION = 4,
       CHARGE_EXCHANGE = 5, CLUSTERING3 = 6 };
enum { SP_E = 0, SP_T2P = 1, SP_T3P = 2, SP_TP = 3 };
enum { R_EXIT0 = 0, R_EXIT1 = 1, R_CUTOFF = 2, R_CAP_COLL = 3, R_CAP_TIME = 4,
       R_RECOMB = 5, R_CLUSTER = 6, R_STALLED = 7 };
enum { DOM_EVENT = 0, DOM_ION_BIRTH = 1, DOM_CLUSTER = 2, DOM_REDRAW = 3, DOM_TARGET = 4 };

/* ---------------- Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11) -------- */
void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
  unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
  *lo = (uint64_t)p;
  *hi = (uint64_t)(p >> 64);
}

void philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
  uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t hi0, lo0, hi1, lo1;
    mulhilo64(M0, x0, &hi0, &lo0);
    mulhilo64(M1, x2, &hi1, &lo1);
    uint64_t y0 = hi1 ^ x1 ^ k0;
    uint64_t y1 = lo1;
    uint64_t y2 = hi0 ^ x3 ^ k1;
    uint64_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += W0; k1 += W1;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* uniform in [0,1) and in (0,1] from the top 53 bits of a word */
double u01(uint64_t w) { return (double)(w >> 11) * (1.0 / 9007199254740992.0); }
double eta01(uint64_t w) { return (double)((w >> 11) + 1) * (1.0 / 9007199254740992.0); }

/* SplitMix64 output function (Steele, Lea, Flood 2014) for lineage ids */
uint64_t mix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
uint64_t child_node(uint64_t parent, uint32_t ev, uint32_t slot) {
  return mix64(mix64(parent) ^ (((uint64_t)ev << 2) | slot));
}

int64_t quant_e(double e_ev) { return (int64_t)std::floor(e_ev * Q_ENERGY); }
/* an energy transfer, rounded to the nearest 2^-24 eV unit */
int64_t quant_recoil(double de_ev) { return (int64_t)std::floor(de_ev * Q_ENERGY + 0.5); }

/* cos(chi) of an elastic collision (Sec. 3.3 Elastic): isotropic (2u - 1)
 * without a table or below the table's threshold energy; otherwise the
 * impact-energy bin of the set is chosen (log-spaced bins, clamped at both
 * ends) and cos chi drawn from its piecewise-linear pdf p on the nodes
 * x_i = -1 + i h: with the cumulative integral C(x), find the interval
 * [x_i, x_i+1] holding t = u C(1) and solve C(x_i) + p_i s + (p_i+1 - p_i)
 * s^2 / 2h = t for s in [0, h]. */
double sample_angle(const orc_problem* p, int ch, double e_imp, double u) {
  const int set = p->ang_set ? p->ang_set[ch] : -1;
  if (set < 0 || !(e_imp >= p->ang_threshold_ev[set])) return 2.0 * u - 1.0;
  const int nb = p->ang_n_bins, n = p->ang_n_mu;
  const double lo = p->ang_e_min_ev[set], hi = p->ang_e_max_ev[set];
  int b = (int)std::floor(std::log(e_imp / lo) / std::log(hi / lo) * nb);
  if (b < 0) b = 0;
  if (b > nb - 1) b = nb - 1;
  const double* pdf = p->ang_pdf + ((size_t)set * nb + b) * n;
  const double h = 2.0 / (double)(n - 1);
  std::vector<double> cum(n, 0.0);
  for (int i = 0; i + 1 < n; ++i) cum[i + 1] = cum[i] + 0.5 * h * (pdf[i] + pdf[i + 1]);
  const double t = u * cum[n - 1];
  int i = 0;
  while (i < n - 2 && cum[i + 1] <= t) ++i;
  const double r = t - cum[i];
  const double a = pdf[i], slope = (pdf[i + 1] - pdf[i]) / h;
  const double disc = std::fmax(0.0, a * a + 2.0 * slope * r);
  const double den = a + std::sqrt(disc);
  double sv = den > 0.0 ? 2.0 * r / den : 0.0;
  sv = std::fmin(std::fmax(sv, 0.0), h);
  return std::fmin(1.0, -1.0 + (double)i * h + sv);
}

/* The block of target-velocity draws number k of one collision (two per
 * attempt of the rejection below). */
typedef void (*TargetBlock)(void* ctx, uint64_t k, uint64_t w[4]);

/* Velocity of the target of an elastic collision (Sec. 3.3 Elastic: the gas
 * drift plus a draw from the Maxwell-Boltzmann distribution at the gas
 * temperature).  Targets of velocity v2 are met at a rate proportional to the
 * relative speed |v1 - v2|, so in the gas frame (impactor velocity u = v1 -
 * drift) the thermal part w is drawn from |u - w| f(w), f the Maxwellian with
 * per-component variance a^2 = kT/M, by the free-gas rejection method: the
 * speed s = |w| from the mixture (|u| + s) s^2 exp(-s^2 / 2a^2) -- with
 * probability |u| sqrt(pi) / (|u| sqrt(pi) + 2 sqrt(2) a) a Maxwell speed
 * (s^2 / a^2 chi-square with 3 degrees of freedom), otherwise s^2 / 2a^2 ~
 * Gamma(2, 1) -- and an isotropic direction, accepted with probability
 * |u - w| / (|u| + s).  Attempt k uses blocks 2k and 2k + 1; after 64
 * rejections the last draw stands.  Velocities in units of c. */
void target_velocity(const orc_problem* p, const double v1[3], TargetBlock blk, void* ctx,
                     double v2[3]) {
  const double a = std::sqrt(KB_EV * p->gas_temperature_k / p->target_mass_ev);
  const double ud = p->gas_drift_mps / C_LIGHT;
  const double u[3] = {v1[0], v1[1], v1[2] - ud};
  const double un = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  const double pmax = un * std::sqrt(M_PI) / (un * std::sqrt(M_PI) + 2.0 * std::sqrt(2.0) * a);
  double w[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < 64; ++k) {
    uint64_t b0[4], b1[4];
    blk(ctx, 2 * (uint64_t)k, b0);
    blk(ctx, 2 * (uint64_t)k + 1, b1);
    const double l1 = -std::log(eta01(b0[1])), l2 = -std::log(eta01(b0[2]));
    double s2;
    if (u01(b0[0]) < pmax) {
      const double c = std::cos(TWO_PI * u01(b0[3]));
      s2 = a * a * (2.0 * l1 + 2.0 * l2 * c * c);       /* chi-square, 3 dof */
    } else {
      s2 = 2.0 * a * a * (l1 + l2);                      /* Gamma(2, 1) */
    }
    const double sp = std::sqrt(s2);
    const double ct = 2.0 * u01(b1[0]) - 1.0;
    const double st = std::sqrt(std::fmax(0.0, 1.0 - ct * ct));
    const double ph = TWO_PI * u01(b1[1]);
    w[0] = sp * st * std::cos(ph);
    w[1] = sp * st * std::sin(ph);
    w[2] = sp * ct;
    const double g0 = u[0] - w[0], g1 = u[1] - w[1], g2 = u[2] - w[2];
    const double gn = std::sqrt(g0 * g0 + g1 * g1 + g2 * g2);
    if (u01(b1[2]) * (un + sp) < gn) break;
  }
  v2[0] = w[0];
  v2[1] = w[1];
  v2[2] = ud + w[2];
}

/* Elastic collision with a moving target (Sec. 3.3 Elastic).  The impactor
 * velocity v1 = sqrt(2E/m1) (sin, 0, cos of the pitch) -- nonrelativistic,
 * gyrophase 0, which loses nothing because the target distribution is
 * symmetric about z.  In the centre-of-mass frame the relative velocity
 * g = v1 - v2 keeps its length and turns by a polar angle chi with cos chi
 * uniform in [-1, 1) (w[2]) and an azimuth 2 pi u (w[3]) measured from the
 * plane of z and g; the impactor leaves with V + m2/(m1+m2) g'.  Velocities in
 * units of c.  v (optional, 12 values): impactor and target before, impactor
 * and target after. */
void moving_target_elastic(const orc_problem* p, int ch, double m1, double e, double mu,
                           const uint64_t w[4], TargetBlock blk, void* ctx, double* e_out,
                           double* mu_out, double* v) {
  const double m2 = p->target_mass_ev;
  const double M = m1 + m2;
  const double s1 = std::sqrt(2.0 * e / m1);
  const double sperp = std::sqrt(std::fmax(0.0, 1.0 - mu * mu));
  const double v1[3] = {s1 * sperp, 0.0, s1 * mu};
  double v2[3];
  target_velocity(p, v1, blk, ctx, v2);
  double V[3], g[3];
  for (int i = 0; i < 3; ++i) {
    V[i] = (m1 * v1[i] + m2 * v2[i]) / M;
    g[i] = v1[i] - v2[i];
  }
  const double gn = std::sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
  double gh[3] = {0.0, 0.0, 1.0};
  if (gn > 0.0) for (int i = 0; i < 3; ++i) gh[i] = g[i] / gn;
  /* e1: the part of z perpendicular to g (x if g is along z), e2 = gh x e1 */
  double e1[3] = {-gh[2] * gh[0], -gh[2] * gh[1], 1.0 - gh[2] * gh[2]};
  double n1 = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
  if (n1 < 1e-12) {
    e1[0] = 1.0; e1[1] = 0.0; e1[2] = 0.0;
    n1 = 1.0;
  }
  for (int i = 0; i < 3; ++i) e1[i] /= n1;
  const double e2[3] = {gh[1] * e1[2] - gh[2] * e1[1], gh[2] * e1[0] - gh[0] * e1[2],
                        gh[0] * e1[1] - gh[1] * e1[0]};
  /* impact energy: the impactor's kinetic energy relative to the target */
  const double cchi = sample_angle(p, ch, 0.5 * m1 * gn * gn, u01(w[2]));
  const double schi = std::sqrt(std::fmax(0.0, 1.0 - cchi * cchi));
  const double phi = TWO_PI * u01(w[3]);
  const double cph = std::cos(phi), sph = std::sin(phi);
  double g2[3], v1n[3];
  for (int i = 0; i < 3; ++i) {
    g2[i] = gn * (schi * cph * e1[i] + schi * sph * e2[i] + cchi * gh[i]);
    v1n[i] = V[i] + m2 / M * g2[i];
  }
  const double sp2 = v1n[0] * v1n[0] + v1n[1] * v1n[1] + v1n[2] * v1n[2];
  *e_out = 0.5 * m1 * sp2;
  *mu_out = sp2 > 0.0 ? std::fmax(-1.0, std::fmin(1.0, v1n[2] / std::sqrt(sp2))) : 1.0;
  if (v) {
    for (int i = 0; i < 3; ++i) {
      v[i] = v1[i];
      v[3 + i] = v2[i];
      v[6 + i] = v1n[i];
      v[9 + i] = V[i] - m1 / M * g2[i];
    }
  }
}

/* Charge exchange (Sec. 3.3 Charge exchange): the impactor of rest energy m1,
 * kinetic energy e and pitch cosine mu takes the velocity of a target
 * particle drawn as for a moving elastic target (target_velocity); its new
 * kinetic energy is 1/2 m1 |v2|^2 and its pitch cosine v2_z / |v2|. */
void charge_exchange(const orc_problem* p, double m1, double e, double mu, TargetBlock blk,
                     void* ctx, double* e_out, double* mu_out, double v2[3]) {
  const double s1 = std::sqrt(2.0 * e / m1);
  const double sperp = std::sqrt(std::fmax(0.0, 1.0 - mu * mu));
  const double v1[3] = {s1 * sperp, 0.0, s1 * mu};
  target_velocity(p, v1, blk, ctx, v2);
  const double sp2 = v2[0] * v2[0] + v2[1] * v2[1] + v2[2] * v2[2];
  *e_out = 0.5 * m1 * sp2;
  *mu_out = sp2 > 0.0 ? std::fmax(-1.0, std::fmin(1.0, v2[2] / std::sqrt(sp2))) : 1.0;
}

/* Target-velocity blocks of redraw r: blocks 128 r + k of the collision's
 * target stream (each target_velocity call reads at most 128 blocks). */
struct RedrawCtx {
  TargetBlock inner;
  void* inner_ctx;
  uint64_t base;
};
void redraw_block(void* c, uint64_t k, uint64_t out[4]) {
  RedrawCtx* q = (RedrawCtx*)c;
  q->inner(q->inner_ctx, q->base + k, out);
}

/* Outcome of an ionization with a moving target: kinetic energies (eV) and
 * pitch cosines of the impactor, the ejected electron and the ion, and the
 * impact energy E_i. */
struct IonOut {
  double e1, mu1, e2, mu2, eion, muion, ei;
};

/* Ionization with a moving target (Sec. 3.3 Ionization).  The target
 * velocity v2 is drawn as for a moving elastic target (target_velocity);
 * while the impact energy -- the impactor's kinetic energy relative to the
 * target, E_i = 1/2 m1 |v1 - v2|^2 -- is not above the ionization energy I, a
 * new target velocity is drawn (redraw r reads blocks 128 r + k; after 64
 * redraws the target is taken at rest, whose impact energy is the lab energy,
 * above I because the channel was chosen).  In the target's frame E_i is
 * shared as for a target at rest: the ejected electron gets W from the
 * truncated 1/(1 + (W/eps)^2) law on [0, (E_i - I)/2] (u = w[2]), the
 * impactor E_i - I - W; their polar angles about the relative velocity are
 * the binary-encounter ones, cos^2 = energy / (E_i - I), at azimuths phi
 * (w[3]) and phi - pi measured from the plane of z and the relative velocity.
 * Adding v2 takes both back to the lab; the ion leaves with v2 (no recoil).
 * Nonrelativistic velocities in units of c, impactor gyrophase 0 (the target
 * distribution is symmetric about z). */
void moving_target_ionization(const orc_problem* p, int ch, double m1, double e, double mu,
                              double m_ion, const uint64_t w[4], TargetBlock blk, void* ctx,
                              IonOut* o) {
  const double me = p->species_mass_ev[SP_E];
  const double ion_e = p->loss_ev[ch];
  const double s1 = std::sqrt(2.0 * e / m1);
  const double sperp = std::sqrt(std::fmax(0.0, 1.0 - mu * mu));
  const double v1[3] = {s1 * sperp, 0.0, s1 * mu};
  double v2[3] = {0.0, 0.0, 0.0}, g[3] = {v1[0], v1[1], v1[2]};
  double ei = e;
  for (int r = 0; r < 64; ++r) {
    RedrawCtx rc = {blk, ctx, 128 * (uint64_t)r};
    double t[3];
    target_velocity(p, v1, redraw_block, &rc, t);
    const double d[3] = {v1[0] - t[0], v1[1] - t[1], v1[2] - t[2]};
    const double er = 0.5 * m1 * (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (er > ion_e) {
      for (int i = 0; i < 3; ++i) { v2[i] = t[i]; g[i] = d[i]; }
      ei = er;
      break;
    }
  }
  /* energy sharing in the target's frame */
  const double avail = ei - ion_e;
  const double eps = p->ioniz_eps_ev;
  const double wmax = 0.5 * avail;
  double wsec = eps * std::tan(u01(w[2]) * std::atan(wmax / eps));
  wsec = std::fmin(std::fmax(wsec, 0.0), wmax);
  const double e1 = avail - wsec;
  const double cp = std::sqrt(e1 / avail), sp = std::sqrt(wsec / avail);
  /* basis: gh along the relative velocity, b1 the part of z perpendicular to
     it (x if it is along z), b2 = gh x b1 */
  const double gn = std::sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
  double gh[3] = {0.0, 0.0, 1.0};
  if (gn > 0.0) for (int i = 0; i < 3; ++i) gh[i] = g[i] / gn;
  double b1[3] = {-gh[2] * gh[0], -gh[2] * gh[1], 1.0 - gh[2] * gh[2]};
  double n1 = std::sqrt(b1[0] * b1[0] + b1[1] * b1[1] + b1[2] * b1[2]);
  if (n1 < 1e-12) { b1[0] = 1.0; b1[1] = 0.0; b1[2] = 0.0; n1 = 1.0; }
  for (int i = 0; i < 3; ++i) b1[i] /= n1;
  const double b2[3] = {gh[1] * b1[2] - gh[2] * b1[1], gh[2] * b1[0] - gh[0] * b1[2],
                        gh[0] * b1[1] - gh[1] * b1[0]};
  const double phi = TWO_PI * u01(w[3]);
  const double cph = std::cos(phi), sph = std::sin(phi);
  const double u1 = std::sqrt(2.0 * e1 / m1), u2 = std::sqrt(2.0 * wsec / me);
  double va[3], vb[3];
  for (int i = 0; i < 3; ++i) {
    const double side = cph * b1[i] + sph * b2[i];
    va[i] = v2[i] + u1 * (cp * gh[i] + sp * side);        /* impactor */
    vb[i] = v2[i] + u2 * (sp * gh[i] - cp * side);        /* ejected electron (phi - pi) */
  }
  const double qa = va[0] * va[0] + va[1] * va[1] + va[2] * va[2];
  const double qb = vb[0] * vb[0] + vb[1] * vb[1] + vb[2] * vb[2];
  const double q2 = v2[0] * v2[0] + v2[1] * v2[1] + v2[2] * v2[2];
  o->e1 = 0.5 * m1 * qa;
  o->mu1 = qa > 0.0 ? std::fmax(-1.0, std::fmin(1.0, va[2] / std::sqrt(qa))) : 1.0;
  o->e2 = 0.5 * me * qb;
  o->mu2 = qb > 0.0 ? std::fmax(-1.0, std::fmin(1.0, vb[2] / std::sqrt(qb))) : 1.0;
  o->eion = 0.5 * m_ion * q2;
  o->muion = q2 > 0.0 ? std::fmax(-1.0, std::fmin(1.0, v2[2] / std::sqrt(q2))) : 1.0;
  o->ei = ei;
}

struct Particle {
  double z;
  int64_t eq;        /* kinetic energy, 2^-24 eV */
  double mu;         /* cos(pitch) w.r.t. +z */
  uint64_t node;     /* lineage id */
  double t_alive;
  uint32_t ev;       /* collisions so far = index of the next flight */
  int species;
};

/* Raw tallies of one worker. */
struct Tally {
  std::vector<uint64_t> spectrum, time_fx, cross_pos, cross_neg, recomb, chan_count;
  std::vector<int64_t> ledger;
  void init(const orc_problem* p) {
    int nz = p->n_zbins;
    spectrum.assign((size_t)2 * ORC_N_SPECIES * (p->n_spec_bins + 1), 0);
    time_fx.assign((size_t)ORC_N_SPECIES * (nz + 2) * p->n_tebins, 0);
    cross_pos.assign((size_t)ORC_N_SPECIES * (nz + 1), 0);
    cross_neg.assign((size_t)ORC_N_SPECIES * (nz + 1), 0);
    recomb.assign((size_t)ORC_N_SPECIES * nz, 0);
    chan_count.assign((size_t)p->n_channels, 0);
    ledger.assign(ORC_LEDGER_LEN, 0);
  }
};

struct Run {
  const orc_problem* p;
  uint64_t seed;
  int pass;          /* 1 or 2 */
  int mode;          /* 0 optical depth, 1 segment stop */
  double dz;
  /* per recombination channel: rate density of the partner field per segment
   * (pass 2 only); electrons use sigma_k(E) * f, ions use f / v. */
  std::vector<std::vector<double>> field;   /* [n_channels][n_zbins] (empty if unused) */
};

double face(const Run& R, int k) {
  return k >= R.p->n_zbins ? R.p->length_m : (double)k * R.dz;
}
int segment_of(const Run& R, double z) {
  int j = (int)std::floor(z / R.dz);
  if (j < 0) j = 0;
  if (j > R.p->n_zbins - 1) j = R.p->n_zbins - 1;
  return j;
}

/* relativistic speed from kinetic energy (Sec. 3.1 remark on gamma) */
double speed(double e_ev, double m_ev) {
  double x = e_ev / m_ev;
  return C_LIGHT * std::sqrt(x * (2.0 + x)) / (1.0 + x);
}

/* cross section of channel k at lab energy E: linear in ln E between nodes */
double sigma_at(const orc_problem* p, int k, double e) {
  if (!(e > p->loss_ev[k])) return 0.0;
  int n = p->n_energy;
  double h = std::log(p->e_max_ev / p->e_min_ev) / (double)(n - 1);
  double x = std::log(e / p->e_min_ev) / h;
  int i = (int)std::floor(x);
  double f;
  if (i < 0) { i = 0; f = 0.0; }
  else if (i > n - 2) { i = n - 2; f = 1.0; }
  else { f = x - (double)i; }
  const double* s = p->sigma_m2 + (size_t)k * n;
  return (1.0 - f) * s[i] + f * s[i + 1];
}

bool channel_active(const Run& R, int k, int species) {
  const orc_problem* p = R.p;
  if (p->species_in[k] != species) return false;
  if (p->kind[k] == RECOMBINATION) return R.pass == 2 && !R.field[k].empty();
  return true;
}

/* Per-flight coefficient of channel k: sigma_k(E) for gas channels and for an
 * electron recombining with an ion field; 1/v for an ion recombining with the
 * electron field (whose per-segment value already carries sigma v).  E is
 * constant along a flight, so these are evaluated once per flight. */
void flight_coefficients(const Run& R, int species, double e, double v, double* c) {
  const orc_problem* p = R.p;
  for (int k = 0; k < p->n_channels; ++k) {
    if (!channel_active(R, k, species)) { c[k] = 0.0; continue; }
    if (p->kind[k] == RECOMBINATION && species != SP_E) c[k] = 1.0 / v;
    else c[k] = sigma_at(p, k, e);
  }
}

/* macroscopic rate per unit path length of channel k in segment j
 * (the inverse mean free path of Eq. mean_free_path, one term); three-body
 * clustering meets two gas molecules, so its rate goes with n^2 */
double channel_rate(const Run& R, int k, const double* c, int j) {
  if (R.p->kind[k] == RECOMBINATION) return R.field[k].empty() ? 0.0 : c[k] * R.field[k][j];
  const double n = R.p->n_seg_m3[j];
  if (R.p->kind[k] == CLUSTERING3) return c[k] * n * n;
  return c[k] * n;
}

double total_rate(const Run& R, const double* c, int j) {
  double r = 0.0;
  for (int k = 0; k < R.p->n_channels; ++k) r += channel_rate(R, k, c, j);
  return r;
}

int tebin(const orc_problem* p, double e) {
  if (p->n_tebins <= 1) return 0;
  double x = std::log(e / p->e_min_ev) / std::log(p->e_max_ev / p->e_min_ev) * p->n_tebins;
  int b = (int)std::floor(x);
  if (b < 0) b = 0;
  if (b > p->n_tebins - 1) b = p->n_tebins - 1;
  return b;
}

uint64_t quant_t(double len, double inv_speed_z) {
  double t = len * inv_speed_z;
  return (uint64_t)(t * Q_TIME + 0.5);
}

struct Worker {
  const Run* R;
  Tally T;
  uint64_t pid;
  uint64_t tree_collisions;

  void add_time(int s, int j, int b, uint64_t q) {
    const orc_problem* p = R->p;
    T.time_fx[((size_t)s * (p->n_zbins + 2) + (j + 1)) * p->n_tebins + b] += q;
  }
  void die(const Particle& P, int reason, int ledger_slot) {
    T.ledger[ORC_DEATHS + P.species * ORC_N_REASONS + reason] += 1;
    T.ledger[ledger_slot] += P.eq;
  }
  void block(uint32_t ev, uint64_t node, int domain, uint64_t sub, uint64_t w[4]) {
    uint64_t ctr[4] = {(uint64_t)ev, node, ((uint64_t)R->pass << 8) | (uint64_t)domain, sub};
    uint64_t key[2] = {R->seed, pid};
    philox4x64_10(ctr, key, w);
  }
  /* thermal target: Gamma(3/2, kT) energy = Exp(1) + Z^2/2 (Box-Muller), isotropic */
  void thermal(const uint64_t w[4], double* e, double* mu) {
    double kt = KB_EV * R->p->gas_temperature_k;
    double c = std::cos(TWO_PI * u01(w[2]));
    *e = kt * (-std::log(eta01(w[0])) - std::log(eta01(w[1])) * c * c);
    *mu = 2.0 * u01(w[3]) - 1.0;
  }

  /* Tally the straight flight z0 -> z1 (both inside [0,L]), direction sign dir. */
  void tally_flight(const Particle& P, double z0, double z1, int dir, double inv_speed_z,
                    int b, bool exits, int jc) {
    const orc_problem* p = R->p;
    int s = P.species;
    int nz = p->n_zbins;
    int j0 = segment_of(*R, z0);
    if (dir > 0) {
      int j1 = exits ? nz - 1 : jc;
      if (j1 < j0) j1 = j0;
      for (int j = j0; j <= j1; ++j) {
        double lo = (j == j0) ? z0 : face(*R, j);
        double hi = (j == j1) ? z1 : face(*R, j + 1);
        bool full = (j != j0) && (j != j1 || exits);
        double len = full ? R->dz : std::fmax(hi - lo, 0.0);
        add_time(s, j, b, quant_t(len, inv_speed_z));
        if (j != j1 || exits) T.cross_pos[(size_t)s * (nz + 1) + j + 1] += 1;
      }
    } else {
      int j1 = exits ? 0 : jc;
      if (j1 > j0) j1 = j0;
      for (int j = j0; j >= j1; --j) {
        double hi = (j == j0) ? z0 : face(*R, j + 1);
        double lo = (j == j1) ? z1 : face(*R, j);
        bool full = (j != j0) && (j != j1 || exits);
        double len = full ? R->dz : std::fmax(hi - lo, 0.0);
        add_time(s, j, b, quant_t(len, inv_speed_z));
        if (j != j1 || exits) T.cross_neg[(size_t)s * (nz + 1) + j] += 1;
      }
    }
  }

  /* Free flight, optical-depth form: walk the segments along the path,
   * accumulating the optical depth until it reaches tau. Returns the end
   * position; *exit_end = 0/1 if the particle left through z=0 / z=L. */
  double flight_optical_depth(const Particle& P, double tau, const double* c, int* exit_end,
                              int* jc) {
    const orc_problem* p = R->p;
    int nz = p->n_zbins;
    double amu = std::fabs(P.mu);
    int dir = P.mu > 0 ? 1 : -1;
    double pos = P.z;
    int j = segment_of(*R, pos);
    double rem = tau;
    for (;;) {
      double r = total_rate(*R, c, j);
      double bound = dir > 0 ? face(*R, j + 1) : face(*R, j);
      double len = dir > 0 ? std::fmax(bound - pos, 0.0) : std::fmax(pos - bound, 0.0);
      double depth = r * len / amu;
      if (r > 0.0 && depth >= rem) {
        double dzc = rem / r * amu;
        double zc = dir > 0 ? pos + dzc : pos - dzc;
        if (dir > 0 && zc > bound) zc = bound;
        if (dir < 0 && zc < bound) zc = bound;
        *exit_end = -1;
        *jc = j;
        return zc;
      }
      rem -= depth;
      if (dir > 0 && j == nz - 1) { *exit_end = 1; return p->length_m; }
      if (dir < 0 && j == 0) { *exit_end = 0; return 0.0; }
      pos = bound;
      j += dir;
    }
  }

  /* Free flight, paper-literal form (Sec. 3.1): in each segment draw a
   * distance from the local mean free path; if it reaches the segment face,
   * stop there without interaction and draw a new distance. */
  double flight_segment_stop(const Particle& P, double eta0, const double* c, int* exit_end,
                             int* jc) {
    const orc_problem* p = R->p;
    int nz = p->n_zbins;
    double amu = std::fabs(P.mu);
    int dir = P.mu > 0 ? 1 : -1;
    double pos = P.z;
    int j = segment_of(*R, pos);
    double eta = eta0;
    uint64_t redraw = 0;
    for (;;) {
      double r = total_rate(*R, c, j);
      double path = r > 0.0 ? -std::log(eta) / r : INFINITY;     /* Eq. distance_from_mfp */
      double bound = dir > 0 ? face(*R, j + 1) : face(*R, j);
      double len = dir > 0 ? std::fmax(bound - pos, 0.0) : std::fmax(pos - bound, 0.0);
      if (path * amu < len) {
        *exit_end = -1;
        *jc = j;
        double zc = dir > 0 ? pos + path * amu : pos - path * amu;
        return zc;
      }
      if (dir > 0 && j == nz - 1) { *exit_end = 1; return p->length_m; }
      if (dir < 0 && j == 0) { *exit_end = 0; return 0.0; }
      pos = bound;
      j += dir;
      uint64_t w[4];
      block(P.ev, P.node, DOM_REDRAW, ++redraw, w);
      eta = eta01(w[0]);
    }
  }

  void spectrum_add(int end, const Particle& P) {
    const orc_problem* p = R->p;
    int64_t binq = (int64_t)std::llround(p->spec_bin_ev * Q_ENERGY);
    int64_t bin = P.eq / binq;
    if (bin > p->n_spec_bins) bin = p->n_spec_bins;
    T.spectrum[((size_t)end * ORC_N_SPECIES + P.species) * (p->n_spec_bins + 1) + bin] += 1;
  }

  /* Follow one particle to termination; products go on the stack. */
  void transport(Particle P, std::vector<Particle>& stack) {
    const orc_problem* p = R->p;
    const int64_t ecut_q = quant_e(p->e_cut_ev);
    std::vector<double> coef((size_t)p->n_channels + 1, 0.0);
    for (;;) {
      /* a particle without kinetic energy never moves: stalled */
      if (P.eq <= 0) { die(P, R_STALLED, ORC_E_STALLED); return; }
      int s = P.species;
      double m = p->species_mass_ev[s];
      double e = (double)P.eq / Q_ENERGY;
      double v = speed(e, m);
      uint64_t w[4];
      block(P.ev, P.node, DOM_EVENT, 0, w);
      double eta = eta01(w[0]);
      double tau = -std::log(eta);                 /* Eq. distance_from_mfp, in optical depth */
      T.ledger[ORC_N_FLIGHTS] += 1;
      T.ledger[ORC_N_FLIGHTS_ALL] += 1;
      flight_coefficients(*R, s, e, v, coef.data());
      int b = tebin(p, e);
      double amu = std::fabs(P.mu);
      double zc;
      int exit_end = -1;
      int j = -1;
      double tflight;
      if (P.mu == 0.0) {
        /* no motion along z: collide in place after path tau / rate */
        j = segment_of(*R, P.z);
        double r = total_rate(*R, coef.data(), j);
        if (!(r > 0.0)) { die(P, R_STALLED, ORC_E_STALLED); return; }
        double path = tau / r;
        tflight = path / v;
        add_time(s, j, b, (uint64_t)(tflight * Q_TIME + 0.5));
        zc = P.z;
      } else {
        if (R->mode == 1) zc = flight_segment_stop(P, eta, coef.data(), &exit_end, &j);
        else zc = flight_optical_depth(P, tau, coef.data(), &exit_end, &j);
        double inv_speed_z = 1.0 / (amu * v);
        tally_flight(P, P.z, zc, P.mu > 0 ? 1 : -1, inv_speed_z, b, exit_end >= 0, j);
        tflight = std::fabs(zc - P.z) * inv_speed_z;
      }
      P.t_alive += tflight;
      if (exit_end >= 0) {                                  /* left the geometry */
        spectrum_add(exit_end, P);
        die(P, exit_end == 0 ? R_EXIT0 : R_EXIT1, exit_end == 0 ? ORC_E_EXIT0 : ORC_E_EXIT1);
        return;
      }
      P.z = zc;
      /* ---- collision in segment j: channel with probability rate_k / rate_tot ---- */
      P.ev += 1;
      tree_collisions += 1;
      T.ledger[ORC_N_COLLISIONS] += 1;
      T.ledger[ORC_N_COLLISIONS_ALL] += 1;
      double rtot = total_rate(*R, coef.data(), j);
      double target = u01(w[1]) * rtot;
      int ch = -1, last = -1;
      double cum = 0.0;
      for (int k = 0; k < p->n_channels; ++k) {
        double rk = channel_rate(*R, k, coef.data(), j);
        if (!(rk > 0.0)) continue;
        last = k;
        cum += rk;
        if (target < cum) { ch = k; break; }
      }
      if (ch < 0) ch = last;                                 /* rounding at the top end */
      T.chan_count[ch] += 1;
      int kind = p->kind[ch];
      if (kind == ELASTIC && p->target && p->target[ch] == 1) {
        /* moving target: its velocity from blocks of its own domain */
        struct Ctx { Worker* self; uint32_t ev; uint64_t node; } cx = {this, P.ev - 1, P.node};
        auto blk = [](void* c, uint64_t k, uint64_t out[4]) {
          Ctx* q = (Ctx*)c;
          q->self->block(q->ev, q->node, DOM_TARGET, k, out);
        };
        double e1, mu1;
        moving_target_elastic(p, ch, m, e, P.mu, w, blk, &cx, &e1, &mu1, nullptr);
        /* energy given to the gas (negative when the gas heats the impactor) */
        int64_t rq = quant_recoil(e - e1);
        if (rq > P.eq) rq = P.eq;
        T.ledger[ORC_E_LOSS_RECOIL] += rq;
        P.eq -= rq;
        P.mu = mu1;
      } else if (kind == CHARGE_EXCHANGE) {
        /* the impactor leaves with a target particle's velocity */
        struct Ctx { Worker* self; uint32_t ev; uint64_t node; } cx = {this, P.ev - 1, P.node};
        auto blk = [](void* c, uint64_t k, uint64_t out[4]) {
          Ctx* q = (Ctx*)c;
          q->self->block(q->ev, q->node, DOM_TARGET, k, out);
        };
        double e1, mu1, v2[3];
        charge_exchange(p, m, e, P.mu, blk, &cx, &e1, &mu1, v2);
        /* kinetic energy handed to the gas (negative when the ion gains) */
        int64_t rq = quant_recoil(e - e1);
        if (rq > P.eq) rq = P.eq;
        T.ledger[ORC_E_LOSS_RECOIL] += rq;
        P.eq -= rq;
        P.mu = mu1;
      } else if (kind == ELASTIC) {
        /* CM polar angle (isotropic or tabulated); lab energy and polar angle
           for a target at rest, whose impact energy is the lab energy */
        double g = m / p->target_mass_ev;
        double cchi = sample_angle(p, ch, e, u01(w[2]));
        double a = 1.0 + 2.0 * g * cchi + g * g;
        double ct = (cchi + g) / std::sqrt(a);
        /* energy given to the target, E - E' = E 2g(1 - cos chi)/(1+g)^2 */
        int64_t rq = quant_recoil(e * 2.0 * g * (1.0 - cchi) / ((1.0 + g) * (1.0 + g)));
        if (rq > P.eq) rq = P.eq;
        T.ledger[ORC_E_LOSS_RECOIL] += rq;
        P.eq -= rq;
        double st = std::sqrt(std::fmax(0.0, 1.0 - ct * ct));
        double cphi = std::cos(TWO_PI * u01(w[3]));
        double smu = std::sqrt(std::fmax(0.0, 1.0 - P.mu * P.mu));
        P.mu = std::fmax(-1.0, std::fmin(1.0, P.mu * ct + smu * st * cphi));
      } else if (kind == EXCITATION) {
        int64_t lq = quant_e(p->loss_ev[ch]);
        P.eq -= lq;
        T.ledger[ORC_E_LOSS_EXCIT] += lq;
      } else if (kind == IONIZATION && p->target && p->target[ch] == 1) {
        /* moving target: impact energy relative to the target, the lab
           energies of the two electrons and the ion's velocity from it */
        struct Ctx { Worker* self; uint32_t ev; uint64_t node; } cx = {this, P.ev - 1, P.node};
        auto blk = [](void* c, uint64_t k, uint64_t out[4]) {
          Ctx* q = (Ctx*)c;
          q->self->block(q->ev, q->node, DOM_TARGET, k, out);
        };
        const int ion = p->species_out[ch];
        const double m_ion = ion >= 0 ? p->species_mass_ev[ion] : p->target_mass_ev;
        IonOut io;
        moving_target_ionization(p, ch, m, e, P.mu, m_ion, w, blk, &cx, &io);
        const int64_t iq = quant_e(p->loss_ev[ch]);
        const int64_t eq1 = quant_e(io.e1), wq = quant_e(io.e2);
        T.ledger[ORC_E_LOSS_IONIZ] += iq;
        /* what the gas gave or took, so the ledger stays exact */
        T.ledger[ORC_E_LOSS_RECOIL] += P.eq - iq - eq1 - wq;
        const uint32_t ev_coll = P.ev - 1;
        Particle S;
        S.z = P.z; S.eq = wq; S.mu = io.mu2; S.node = child_node(P.node, ev_coll, 0);
        S.t_alive = 0.0; S.ev = 0; S.species = SP_E;
        T.ledger[ORC_BIRTHS + SP_E] += 1;
        T.ledger[ORC_N_SPAWN_E] += 1;
        if (S.eq < ecut_q) die(S, R_CUTOFF, ORC_E_CUTOFF);
        else stack.push_back(S);
        if (ion >= 0) {
          Particle I;
          I.z = P.z; I.node = child_node(P.node, ev_coll, 1);
          I.t_alive = 0.0; I.ev = 0; I.species = ion;
          I.eq = quant_e(io.eion); I.mu = io.muion;
          T.ledger[ORC_E_IN_THERMAL] += I.eq;
          T.ledger[ORC_BIRTHS + ion] += 1;
          T.ledger[ORC_N_SPAWN_ION] += 1;
          stack.push_back(I);
        }
        P.eq = eq1;
        P.mu = io.mu1;
      } else if (kind == IONIZATION) {
        int64_t iq = quant_e(p->loss_ev[ch]);
        int64_t avail = P.eq - iq;
        double eps = p->ioniz_eps_ev;
        double wmax = (e - p->loss_ev[ch]) * 0.5;
        double wsec = eps * std::tan(u01(w[2]) * std::atan(wmax / eps));
        int64_t wq = quant_e(wsec);
        if (wq > avail / 2) wq = avail / 2;
        if (wq < 0) wq = 0;
        int64_t eq1 = avail - wq;
        T.ledger[ORC_E_LOSS_IONIZ] += iq;
        double c2p = avail > 0 ? (double)eq1 / (double)avail : 1.0;   /* cos^2 primary */
        double c2s = avail > 0 ? (double)wq / (double)avail : 0.0;    /* cos^2 secondary */
        double cp = std::sqrt(c2p), sp = std::sqrt(c2s);              /* sin_p = cos_s */
        double cphi = std::cos(TWO_PI * u01(w[3]));
        double smu = std::sqrt(std::fmax(0.0, 1.0 - P.mu * P.mu));
        double mu_p = std::fmax(-1.0, std::fmin(1.0, P.mu * cp + smu * sp * cphi));
        double mu_s = std::fmax(-1.0, std::fmin(1.0, P.mu * sp - smu * cp * cphi));
        uint32_t ev_coll = P.ev - 1;
        /* secondary electron */
        Particle S;
        S.z = P.z; S.eq = wq; S.mu = mu_s; S.node = child_node(P.node, ev_coll, 0);
        S.t_alive = 0.0; S.ev = 0; S.species = SP_E;
        T.ledger[ORC_BIRTHS + SP_E] += 1;
        T.ledger[ORC_N_SPAWN_E] += 1;
        if (S.eq < ecut_q) die(S, R_CUTOFF, ORC_E_CUTOFF);
        else stack.push_back(S);
        /* ion with the target's (thermal) velocity */
        int ion = p->species_out[ch];
        if (ion >= 0) {
          Particle I;
          I.z = P.z; I.node = child_node(P.node, ev_coll, 1);
          I.t_alive = 0.0; I.ev = 0; I.species = ion;
          uint64_t wi[4];
          block(0, I.node, DOM_ION_BIRTH, 0, wi);
          double ei, mui;
          thermal(wi, &ei, &mui);
          I.eq = quant_e(ei); I.mu = mui;
          T.ledger[ORC_E_IN_THERMAL] += I.eq;
          T.ledger[ORC_BIRTHS + ion] += 1;
          T.ledger[ORC_N_SPAWN_ION] += 1;
          stack.push_back(I);
        }
        P.eq = eq1;
        P.mu = mu_p;
      } else if (kind == CLUSTERING || kind == CLUSTERING3) {
        /* incident ion consumed; product with a thermal target's energy */
        die(P, R_CLUSTER, ORC_E_CLUSTER);
        uint64_t wc[4];
        block(P.ev - 1, P.node, DOM_CLUSTER, 0, wc);
        double ec, muc;
        thermal(wc, &ec, &muc);
        Particle C;
        C.z = P.z; C.eq = quant_e(ec); C.mu = muc;
        C.node = child_node(P.node, P.ev - 1, 2);
        C.t_alive = 0.0; C.ev = 0; C.species = p->species_out[ch];
        T.ledger[ORC_E_IN_THERMAL] += C.eq;
        T.ledger[ORC_BIRTHS + C.species] += 1;
        P = C;
        continue;
      } else if (kind == RECOMBINATION) {
        int partner = p->species_out[ch];
        T.recomb[(size_t)partner * p->n_zbins + j] += 1;
        die(P, R_RECOMB, ORC_E_RECOMB);
        return;
      }
      /* ---- terminator (Sec. 3.2) ---- */
      if (P.species == SP_E && P.eq < ecut_q) { die(P, R_CUTOFF, ORC_E_CUTOFF); return; }
      if (P.ev >= p->max_collisions) { die(P, R_CAP_COLL, ORC_E_CAP); return; }
      if (P.t_alive >= p->max_lifetime_s) { die(P, R_CAP_TIME, ORC_E_CAP); return; }
    }
  }

  void run_range(const orc_primaries* pr, int64_t lo, int64_t hi, uint64_t* per_primary) {
    const orc_problem* p = R->p;
    const int64_t ecut_q = quant_e(p->e_cut_ev);
    std::vector<Particle> stack;
    for (int64_t i = lo; i < hi; ++i) {
      pid = (uint64_t)(pr->pid_offset + i);
      tree_collisions = 0;
      Particle P;
      P.z = pr->z_m[i]; P.eq = quant_e(pr->e_ev[i]); P.mu = pr->mu[i];
      P.node = 0; P.t_alive = 0.0; P.ev = 0; P.species = pr->species[i];
      T.ledger[ORC_E_IN_PRIMARY] += P.eq;
      T.ledger[ORC_BIRTHS + P.species] += 1;
      if (P.species == SP_E && P.eq < ecut_q) die(P, R_CUTOFF, ORC_E_CUTOFF);
      else stack.push_back(P);
      while (!stack.empty()) {
        Particle Q = stack.back();
        stack.pop_back();
        transport(Q, stack);
      }
      if (per_primary) per_primary[i] += tree_collisions;
    }
  }
};

/* Target fields from summed time tallies and recombination deletions
 * (Eq. target_field_density: n = sum t / (t_sim V) - N_gamma / V, t_sim of
 * Eq. simulated_time over n_decays).  The partner's density in energy bin b
 * of segment j takes its share of the segment's deletions in proportion to
 * its time there; a density below zero counts as zero.  recomb_in NULL: no
 * deletions (the fields of a two-pass run, whose pass 1 has none).
 * Electron impactor: the ion partner's density; ion impactor: the electron
 * field weighted by sigma(E_b) v(E_b) at the bin centres. */
void build_fields(Run& R, const uint64_t* time_in, const uint64_t* recomb_in, double n_decays) {
  const orc_problem* p = R.p;
  int nz = p->n_zbins, ntb = p->n_tebins;
  double tsim = n_decays / p->activity_bq;
  double vol = R.dz * p->area_m2;
  R.field.assign(p->n_channels, std::vector<double>());
  for (int k = 0; k < p->n_channels; ++k) {
    if (p->kind[k] != RECOMBINATION) continue;
    int partner = p->species_out[k];
    std::vector<double> f(nz, 0.0);
    for (int j = 0; j < nz; ++j) {
      const uint64_t* tj = time_in + ((size_t)partner * (nz + 2) + (j + 1)) * ntb;
      double ttot = 0.0;
      for (int b = 0; b < ntb; ++b) ttot += (double)tj[b];
      const double del = recomb_in ? (double)recomb_in[(size_t)partner * nz + j] / vol : 0.0;
      double acc = 0.0;
      for (int b = 0; b < ntb; ++b) {
        double n = (double)tj[b] / Q_TIME / (tsim * vol);
        if (recomb_in && ttot > 0.0) n -= del * ((double)tj[b] / ttot);
        if (p->species_in[k] == SP_E) {
          acc += n;                                  /* ion density */
        } else {
          /* ion impactor: electron field weighted by sigma(E_b) v(E_b) */
          double eb = p->e_min_ev * std::pow(p->e_max_ev / p->e_min_ev, (b + 0.5) / ntb);
          acc += std::fmax(n, 0.0) * sigma_at(p, k, eb) * speed(eb, p->species_mass_ev[SP_E]);
        }
      }
      f[j] = std::fmax(acc, 0.0);
    }
    R.field[k] = f;
  }
}

void add_into(orc_tallies* out, const Tally& T, const orc_problem* p) {
  for (size_t i = 0; i < T.spectrum.size(); ++i) out->spectrum[i] += T.spectrum[i];
  for (size_t i = 0; i < T.time_fx.size(); ++i) out->time_fx[i] += T.time_fx[i];
  for (size_t i = 0; i < T.cross_pos.size(); ++i) out->cross_pos[i] += T.cross_pos[i];
  for (size_t i = 0; i < T.cross_neg.size(); ++i) out->cross_neg[i] += T.cross_neg[i];
  for (size_t i = 0; i < T.recomb.size(); ++i) out->recomb[i] += T.recomb[i];
  for (int i = 0; i < ORC_LEDGER_LEN; ++i) out->ledger[i] += T.ledger[i];
  for (int i = 0; i < p->n_channels; ++i) out->chan_count[i] += T.chan_count[i];
}

int check_problem(const orc_problem* p) {
  if (!p || p->n_zbins <= 0 || !(p->length_m > 0) || p->n_energy < 2 || p->n_channels < 0 ||
      p->n_tebins < 1 || p->n_spec_bins < 1 || !(p->spec_bin_ev > 0) || !p->n_seg_m3)
    return 1;
  return 0;
}

/* One pass.  Pass 2 takes its target fields from field_time_in (and the
 * deletions field_recomb_in, may be NULL) over field_decays decays; with
 * zero_fields the recombination channels are present with fields of zero. */
int do_pass(const orc_problem* p, const orc_primaries* pr, uint64_t seed, int pass,
            const uint64_t* field_time_in, const uint64_t* field_recomb_in, double field_decays,
            bool zero_fields, int mode, int n_threads, orc_tallies* out) {
  Run R;
  R.p = p; R.seed = seed; R.pass = pass; R.mode = mode;
  R.dz = p->length_m / p->n_zbins;
  R.field.assign(p->n_channels, std::vector<double>());
  if (pass == 2 && field_time_in) build_fields(R, field_time_in, field_recomb_in, field_decays);
  if (pass == 2 && zero_fields)
    for (int k = 0; k < p->n_channels; ++k)
      if (p->kind[k] == RECOMBINATION) R.field[k].assign(p->n_zbins, 0.0);
  if (n_threads < 1) n_threads = 1;
  if ((int64_t)n_threads > pr->n) n_threads = (int)(pr->n > 0 ? pr->n : 1);
  std::vector<Worker> W(n_threads);
  std::vector<std::thread> th;
  for (int t = 0; t < n_threads; ++t) {
    W[t].R = &R;
    W[t].T.init(p);
    int64_t lo = pr->n * t / n_threads, hi = pr->n * (t + 1) / n_threads;
    if (n_threads == 1) W[t].run_range(pr, lo, hi, out->per_primary);
    else th.emplace_back([&W, t, pr, lo, hi, out] { W[t].run_range(pr, lo, hi, out->per_primary); });
  }
  for (auto& x : th) x.join();
  for (int t = 0; t < n_threads; ++t) add_into(out, W[t].T, p);
  return 0;
}


/* ======================= orbit mode: Boris mover (Sec. 3.1) =======================
 *
 * Readings: the relativistic form of the Boris push (the paper's equations with
 * the proper velocity u = gamma v, gamma of the half-accelerated velocity in
 * the rotation); the initial velocity is taken as the half-step velocity; the
 * time of a step goes to the z segment and radial bin of the step's midpoint
 * (segment floor(z n_zbins / L); radial bin k for (k R / n_rbins)^2 <= x^2 + y^2
 * < ((k + 1) R / n_rbins)^2, the last bin open above);
 * the optical depth of a step is the total rate of the midpoint's segment
 * times the step's path length; the cross sections are those of the flight's
 * starting energy, and with an electric field a flight also ends, without
 * interaction, after the step in which the kinetic energy leaves its bin of
 * the time tally's energy grid (Sec. 3.1: the movement stops when the
 * particle leaves an energy bin of the density fields and a new distance is
 * drawn); a step that reaches the drawn optical depth, a z end, the wall or
 * the lifetime cap is shortened to the fraction of its displacement where
 * that happens (first of them; on a tie: wall, z end, lifetime, collision). */
const double CHARGE_E[ORC_N_SPECIES] = {-1.0, 1.0, 1.0, 1.0};   /* units of e */
const double INV_C2 = 1.0 / (C_LIGHT * C_LIGHT);
enum { OEV_NONE = 0, OEV_WALL = 1, OEV_EXIT = 2, OEV_CAP = 3, OEV_COLL = 4, OEV_EBIN = 5 };

struct OParticle {
  double x[3];       /* position (m) */
  double u[3];       /* proper velocity gamma v (m/s) */
  uint64_t node;     /* lineage id */
  double t_alive;
  uint32_t ev;       /* collisions so far */
  int species;
};

/* kinetic energy (eV) of proper velocity u: (gamma - 1) m with
 * gamma - 1 = x / (gamma + 1), x = u^2 / c^2 (no cancellation when slow) */
double kinetic_u(const double u[3], double m_ev) {
  double x = (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) / (C_LIGHT * C_LIGHT);
  double g = std::sqrt(1.0 + x);
  return m_ev * x / (g + 1.0);
}

/* proper speed gamma v (m/s) of kinetic energy e: c sqrt(y (2 + y)), y = e / m */
double proper_speed(double e_ev, double m_ev) {
  double y = e_ev / m_ev;
  return C_LIGHT * std::sqrt(y * (2.0 + y));
}

/* The direction at polar angle acos(ct) and azimuth (cp, sp) = (cos, sin)
 * about the unit vector d, in the frame e1 = (z - d_z d) / s (the unit vector
 * normal to d towards +z), e2 = d x e1 = (d_y, -d_x, 0) / s, s = sqrt(d_x^2 +
 * d_y^2); for s below 1e-12, e1 = x, e2 = d x x.  Its z component is then
 * d_z ct + s st cp, the guiding-centre update of the pitch cosine. */
void turn(const double d[3], double ct, double cp, double sp, double out[3]) {
  const double s = std::sqrt(d[0] * d[0] + d[1] * d[1]);
  double e1[3], e2[3];
  if (s > 1e-12) {
    e1[0] = -d[2] * d[0] / s; e1[1] = -d[2] * d[1] / s; e1[2] = s;
    e2[0] = d[1] / s; e2[1] = -d[0] / s; e2[2] = 0.0;
  } else {
    e1[0] = 1.0; e1[1] = 0.0; e1[2] = 0.0;
    e2[0] = 0.0; e2[1] = d[2]; e2[2] = -d[1];
  }
  const double st = std::sqrt(std::fmax(0.0, 1.0 - ct * ct));
  for (int i = 0; i < 3; ++i) out[i] = ct * d[i] + st * (cp * e1[i] + sp * e2[i]);
}

struct OrbitRun {
  const orc_problem* p;
  const orc_orbit* o;
  uint64_t seed;
  double dz;
  double inv_dz;     /* n_zbins / L */
  double r_scale;    /* n_rbins / R */
  std::vector<double> edge2;   /* [n_rbins + 1] squared radii of the radial bin edges */
  bool fields;       /* some electric field is present */
  uint64_t max_steps;
};

struct OTally {
  std::vector<uint64_t> spectrum, time_z, time_r, cross_pos, cross_neg, rcross_out, rcross_in,
      wall, chan_count;
  std::vector<int64_t> ledger;
  std::vector<double> energy;
  void init(const orc_problem* p, const orc_orbit* o) {
    int nz = p->n_zbins, nr = o->n_rbins;
    spectrum.assign((size_t)2 * ORC_N_SPECIES * (p->n_spec_bins + 1), 0);
    time_z.assign((size_t)ORC_N_SPECIES * nz, 0);
    time_r.assign((size_t)ORC_N_SPECIES * nr, 0);
    cross_pos.assign((size_t)ORC_N_SPECIES * (nz + 1), 0);
    cross_neg.assign((size_t)ORC_N_SPECIES * (nz + 1), 0);
    rcross_out.assign((size_t)ORC_N_SPECIES * (nr + 1), 0);
    rcross_in.assign((size_t)ORC_N_SPECIES * (nr + 1), 0);
    wall.assign((size_t)ORC_N_SPECIES * nz, 0);
    chan_count.assign((size_t)p->n_channels, 0);
    ledger.assign(ORC_OB_LEDGER_LEN, 0);
    energy.assign(ORC_OE_LEN, 0.0);
  }
};

struct OWorker {
  const OrbitRun* R;
  OTally T;
  uint64_t pid;
  uint64_t tree_collisions;

  void block(uint32_t ev, uint64_t node, int domain, uint64_t sub, uint64_t w[4]) {
    uint64_t ctr[4] = {(uint64_t)ev, node, (1ULL << 8) | (uint64_t)domain, sub};
    uint64_t key[2] = {R->seed, pid};
    philox4x64_10(ctr, key, w);
  }
  int seg(double z) const {
    int j = (int)std::floor(z * R->inv_dz);
    if (j < 0) j = 0;
    if (j > R->p->n_zbins - 1) j = R->p->n_zbins - 1;
    return j;
  }
  int rbin(double x, double y) const {
    const double q = x * x + y * y;
    const int nr = R->o->n_rbins;
    int b = (int)std::floor(std::sqrt(q) * R->r_scale);     /* a first guess */
    if (b < 0) b = 0;
    if (b > nr - 1) b = nr - 1;
    while (b > 0 && R->edge2[b] > q) --b;
    while (b < nr - 1 && R->edge2[b + 1] <= q) ++b;
    return b;
  }
  void die(const OParticle& P, int reason, int eslot, double e) {
    T.ledger[ORC_OB_DEATHS + P.species * ORC_N_REASONS + reason] += 1;
    T.energy[eslot] += e;
  }
  /* per-flight coefficients sigma_k(E) of the species' channels */
  void coefficients(int s, double e, double* c) const {
    const orc_problem* p = R->p;
    for (int k = 0; k < p->n_channels; ++k)
      c[k] = p->species_in[k] == s ? sigma_at(p, k, e) : 0.0;
  }
  double rate_k(int k, const double* c, int j) const {
    const double n = R->p->n_seg_m3[j];
    return R->p->kind[k] == CLUSTERING3 ? c[k] * n * n : c[k] * n;
  }
  double rate(const double* c, int j) const {
    double r = 0.0;
    for (int k = 0; k < R->p->n_channels; ++k) r += rate_k(k, c, j);
    return r;
  }
  /* rate per unit path of a step in segment j: n_j times the two-body cross
     sections plus n_j^2 times the three-body coefficients */
  double step_rate(const double* c, int j) const {
    double s1 = 0.0, s3 = 0.0;
    for (int k = 0; k < R->p->n_channels; ++k) {
      if (R->p->kind[k] == CLUSTERING3) s3 += c[k];
      else s1 += c[k];
    }
    const double n = R->p->n_seg_m3[j];
    return s1 * n + s3 * (n * n);
  }
  /* thermal product: Gamma(3/2, kT) energy and an isotropic direction */
  void thermal3(uint32_t ev, uint64_t node, int domain, double* e, double d[3]) {
    uint64_t w[4], w2[4];
    block(ev, node, domain, 0, w);
    block(ev, node, domain, 1, w2);
    double kt = KB_EV * R->p->gas_temperature_k;
    double c = std::cos(TWO_PI * u01(w[2]));
    *e = kt * (-std::log(eta01(w[0])) - std::log(eta01(w[1])) * c * c);
    double mu = 2.0 * u01(w[3]);
    mu -= 1.0;
    double st = std::sqrt(std::fmax(0.0, 1.0 - mu * mu));
    double ph = TWO_PI * u01(w2[0]);
    d[0] = st * std::cos(ph);
    d[1] = st * std::sin(ph);
    d[2] = mu;
  }
  void set_u(OParticle& P, double e, const double d[3]) {
    double ps = proper_speed(e, R->p->species_mass_ev[P.species]);
    for (int i = 0; i < 3; ++i) P.u[i] = ps * d[i];
  }
  /* time of a run of steps in one (segment, radial bin) cell */
  void flush(int s, int cj, int cr, uint64_t n_full, double f_last, double dt) {
    if (cj < 0) return;
    double t = (double)n_full * dt + f_last * dt;
    uint64_t q = (uint64_t)(t * Q_TIME + 0.5);
    T.time_z[(size_t)s * R->p->n_zbins + cj] += q;
    T.time_r[(size_t)s * R->o->n_rbins + cr] += q;
  }
  /* crossings of z faces and of the radial bin boundaries by a straight step
   * from a to b (z ends and the wall are counted by the caller) */
  void crossings(int s, const double a[3], const double b[3]) {
    const int nz = R->p->n_zbins, nr = R->o->n_rbins;
    int ja = seg(a[2]), jb = seg(b[2]);
    for (int k = ja + 1; k <= jb; ++k) T.cross_pos[(size_t)s * (nz + 1) + k] += 1;
    for (int k = jb + 1; k <= ja; ++k) T.cross_neg[(size_t)s * (nz + 1) + k] += 1;
    int ra = rbin(a[0], a[1]), rb = rbin(b[0], b[1]);
    for (int k = ra + 1; k <= rb; ++k) T.rcross_out[(size_t)s * (nr + 1) + k] += 1;
    for (int k = rb + 1; k <= ra; ++k) T.rcross_in[(size_t)s * (nr + 1) + k] += 1;
  }
  void spectrum_add(int end, int s, double e) {
    const orc_problem* p = R->p;
    double x = std::floor(e / p->spec_bin_ev);
    int64_t bin = x < 0.0 ? 0 : (x > (double)p->n_spec_bins ? p->n_spec_bins : (int64_t)x);
    T.spectrum[((size_t)end * ORC_N_SPECIES + s) * (p->n_spec_bins + 1) + bin] += 1;
  }
  void write_end(double* es, const OParticle& P) {
    if (!es || P.node != 0) return;
    double e = kinetic_u(P.u, R->p->species_mass_ev[P.species]);
    double v[8] = {P.x[0], P.x[1], P.x[2], e, P.u[0], P.u[1], P.u[2], P.t_alive};
    for (int i = 0; i < 8; ++i) es[i] = v[i];
  }

  /* Follow one particle to its end; products go on the stack. */
  void transport(OParticle P, std::vector<OParticle>& stack, double* es) {
    const orc_problem* p = R->p;
    const orc_orbit* o = R->o;
    const int nz = p->n_zbins, nr = o->n_rbins;
    const double L = p->length_m, R2 = o->tube_radius_m * o->tube_radius_m;
    std::vector<double> coef((size_t)p->n_channels + 1, 0.0);
    uint64_t redraw = 0;             /* flights ended by an energy-bin change since the last event */
    for (;;) {
      const int s = P.species;
      const double m = p->species_mass_ev[s];
      const double e0 = kinetic_u(P.u, m);
      if (!(e0 > 0.0)) { write_end(es, P); die(P, ORC_OR_STALLED, ORC_OE_STALLED, e0); return; }
      /* the collision's uniforms come from the event's block; after an
         energy-bin stop the optical depth is drawn anew from redraw blocks */
      uint64_t w[4];
      block(P.ev, P.node, DOM_EVENT, 0, w);
      double tau = -std::log(eta01(w[0]));
      if (redraw > 0) {
        uint64_t wr[4];
        block(P.ev, P.node, DOM_REDRAW, redraw, wr);
        tau = -std::log(eta01(wr[0]));
      }
      T.ledger[ORC_OB_N_FLIGHTS] += 1;
      coefficients(s, e0, coef.data());
      /* the flight's energy bin as bounds on u^2 (with an electric field) */
      double u2_lo = -1.0, u2_hi = INFINITY;
      if (R->fields) {
        const int b = tebin(p, e0), ntb = p->n_tebins;
        const double ratio = p->e_max_ev / p->e_min_ev;
        if (b > 0) {
          const double ps = proper_speed(p->e_min_ev * std::pow(ratio, (double)b / ntb), m);
          u2_lo = ps * ps;
        }
        if (b < ntb - 1) {
          const double ps = proper_speed(p->e_min_ev * std::pow(ratio, (double)(b + 1) / ntb), m);
          u2_hi = ps * ps;
        }
      }
      const double dt = o->dt_s[s];
      const double h = 0.5 * (CHARGE_E[s] * C_LIGHT * C_LIGHT / m) * dt;   /* q dt / 2m */
      double acc = 0.0;
      int cj = -1, cr = -1;          /* cell of the current run of steps */
      uint64_t cn = 0;
      int event = OEV_NONE, end = -1;
      for (uint64_t step = 0;; ++step) {
        if (step >= R->max_steps) {
          flush(s, cj, cr, cn, 0.0, dt);
          T.energy[ORC_OE_FIELD_WORK] += kinetic_u(P.u, m) - e0;
          write_end(es, P);
          die(P, ORC_OR_STALLED, ORC_OE_STALLED, kinetic_u(P.u, m));
          return;
        }
        T.ledger[ORC_OB_N_STEPS] += 1;
        const double* x = P.x;
        /* Boris push: half electric kick, magnetic rotation, half kick */
        const double ef[3] = {o->e_r_vm2 * x[0], o->e_r_vm2 * x[1],
                              o->e_z_vm ? o->e_z_vm[seg(x[2])] : 0.0};
        double um[3];
        for (int i = 0; i < 3; ++i) um[i] = P.u[i] + h * ef[i];
        const double gm = std::sqrt(1.0 + (um[0] * um[0] + um[1] * um[1] + um[2] * um[2]) * INV_C2);
        const double t = h * o->b_t / gm;
        const double sf = 2.0 * t / (1.0 + t * t);
        const double upx = um[0] + um[1] * t, upy = um[1] - um[0] * t;
        double un[3] = {um[0] + upy * sf, um[1] - upx * sf, um[2]};
        for (int i = 0; i < 3; ++i) un[i] += h * ef[i];
        const double u2n = un[0] * un[0] + un[1] * un[1] + un[2] * un[2];
        const double gn = std::sqrt(1.0 + u2n * INV_C2);
        const double sc = dt / gn;
        const double d[3] = {un[0] * sc, un[1] * sc, un[2] * sc};
        const double ds = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        const int jm = seg(x[2] + 0.5 * d[2]);
        const double dtau = step_rate(coef.data(), jm) * ds;
        /* the first of wall, z end, lifetime cap and collision within the step */
        double fb = 1.0;
        event = OEV_NONE;
        const double xn = x[0] + d[0], yn = x[1] + d[1], zn = x[2] + d[2];
        if (xn * xn + yn * yn > R2) {
          /* |p + f q|^2 = R^2 for the transverse parts p, q: the root in (0, 1] */
          const double a = d[0] * d[0] + d[1] * d[1];
          const double b = x[0] * d[0] + x[1] * d[1];
          const double c = x[0] * x[0] + x[1] * x[1] - R2;
          const double disc = std::sqrt(std::fmax(0.0, b * b - a * c));
          double f = b > 0.0 ? -c / (b + disc) : (disc - b) / a;
          f = std::fmin(1.0, std::fmax(0.0, f));
          if (f <= fb) { fb = f; event = OEV_WALL; }
        }
        if (zn < 0.0 || zn > L) {
          double f = zn < 0.0 ? -x[2] / d[2] : (L - x[2]) / d[2];
          f = std::fmin(1.0, std::fmax(0.0, f));
          if (event == OEV_NONE ? f <= fb : f < fb) { fb = f; event = OEV_EXIT; end = zn < 0.0 ? 0 : 1; }
        }
        if (P.t_alive + dt >= p->max_lifetime_s) {
          double f = std::fmin(1.0, std::fmax(0.0, (p->max_lifetime_s - P.t_alive) / dt));
          if (event == OEV_NONE ? f <= fb : f < fb) { fb = f; event = OEV_CAP; }
        }
        if (dtau > 0.0 && acc + dtau >= tau) {
          double f = std::fmin(1.0, std::fmax(0.0, (tau - acc) / dtau));
          if (event == OEV_NONE ? f <= fb : f < fb) { fb = f; event = OEV_COLL; }
        }
        if (event == OEV_NONE && (u2n < u2_lo || u2n >= u2_hi)) event = OEV_EBIN;
        if (event == OEV_NONE || event == OEV_EBIN) {
          const int mj = jm, mr = rbin(x[0] + 0.5 * d[0], x[1] + 0.5 * d[1]);
          if (mj == cj && mr == cr) {
            cn += 1;
          } else {
            flush(s, cj, cr, cn, 0.0, dt);
            cj = mj; cr = mr; cn = 1;
          }
          const double b[3] = {xn, yn, zn};
          crossings(s, x, b);
          P.x[0] = xn; P.x[1] = yn; P.x[2] = zn;
          P.t_alive += dt;
          acc += dtau;
          for (int i = 0; i < 3; ++i) P.u[i] = un[i];
          if (event == OEV_NONE) continue;
          flush(s, cj, cr, cn, 0.0, dt);       /* left the energy bin: a new flight */
          break;
        }
        /* the shortened last step */
        const double dp[3] = {fb * d[0], fb * d[1], fb * d[2]};
        const int mj = seg(x[2] + 0.5 * dp[2]), mr = rbin(x[0] + 0.5 * dp[0], x[1] + 0.5 * dp[1]);
        if (mj == cj && mr == cr) {
          flush(s, cj, cr, cn, fb, dt);
        } else {
          flush(s, cj, cr, cn, 0.0, dt);
          flush(s, mj, mr, 0, fb, dt);
        }
        double b[3] = {x[0] + dp[0], x[1] + dp[1], x[2] + dp[2]};
        if (event == OEV_EXIT) b[2] = end == 0 ? 0.0 : L;
        crossings(s, x, b);
        P.x[0] = b[0]; P.x[1] = b[1]; P.x[2] = b[2];
        P.t_alive = event == OEV_CAP ? p->max_lifetime_s : P.t_alive + fb * dt;
        for (int i = 0; i < 3; ++i) P.u[i] = un[i];
        break;
      }
      const double e1 = kinetic_u(P.u, m);
      T.energy[ORC_OE_FIELD_WORK] += e1 - e0;
      if (event == OEV_EBIN) { ++redraw; continue; }
      if (event == OEV_WALL) {
        T.wall[(size_t)s * nz + seg(P.x[2])] += 1;
        const int ra = rbin(P.x[0], P.x[1]);
        for (int k = ra + 1; k <= nr; ++k) T.rcross_out[(size_t)s * (nr + 1) + k] += 1;
        write_end(es, P);
        die(P, ORC_OR_WALL, ORC_OE_WALL, e1);
        return;
      }
      if (event == OEV_EXIT) {
        if (end == 1) T.cross_pos[(size_t)s * (nz + 1) + nz] += 1;
        else T.cross_neg[(size_t)s * (nz + 1) + 0] += 1;
        spectrum_add(end, s, e1);
        write_end(es, P);
        die(P, end == 0 ? ORC_OR_EXIT0 : ORC_OR_EXIT1, end == 0 ? ORC_OE_EXIT0 : ORC_OE_EXIT1, e1);
        return;
      }
      if (event == OEV_CAP) {
        write_end(es, P);
        die(P, ORC_OR_CAP_TIME, ORC_OE_CAP, e1);
        return;
      }
      /* ---- collision: channel with probability rate_k / rate_tot ---- */
      const int j = seg(P.x[2]);
      P.ev += 1;
      redraw = 0;
      tree_collisions += 1;
      T.ledger[ORC_OB_N_COLLISIONS] += 1;
      double rtot = rate(coef.data(), j);
      double target = u01(w[1]) * rtot;
      int ch = -1, last = -1;
      double cum = 0.0;
      for (int k = 0; k < p->n_channels; ++k) {
        double rk = rate_k(k, coef.data(), j);
        if (!(rk > 0.0)) continue;
        last = k;
        cum += rk;
        if (target < cum) { ch = k; break; }
      }
      if (ch < 0) ch = last;
      T.chan_count[ch] += 1;
      const int kind = p->kind[ch];
      const double ec = e1;
      const double pu = std::sqrt(P.u[0] * P.u[0] + P.u[1] * P.u[1] + P.u[2] * P.u[2]);
      const double dir[3] = {P.u[0] / pu, P.u[1] / pu, P.u[2] / pu};
      const double ph = TWO_PI * u01(w[3]);
      const double cph = std::cos(ph), sph = std::sin(ph);
      const uint32_t ev_coll = P.ev - 1;
      double enew = ec;
      if (kind == ELASTIC) {
        double g = m / p->target_mass_ev;
        double cchi = sample_angle(p, ch, ec, u01(w[2]));
        double a = 1.0 + 2.0 * g * cchi + g * g;
        double ct = (cchi + g) / std::sqrt(a);
        double loss = ec * 2.0 * g * (1.0 - cchi) / ((1.0 + g) * (1.0 + g));
        enew = ec - loss;
        T.energy[ORC_OE_RECOIL] += loss;
        double nd[3];
        turn(dir, ct, cph, sph, nd);
        set_u(P, enew, nd);
      } else if (kind == EXCITATION) {
        enew = ec - p->loss_ev[ch];
        T.energy[ORC_OE_LOSS_EXCIT] += p->loss_ev[ch];
        set_u(P, enew, dir);
      } else if (kind == IONIZATION) {
        const double ion_e = p->loss_ev[ch];
        const double avail = ec - ion_e;
        const double eps = p->ioniz_eps_ev;
        double wsec = eps * std::tan(u01(w[2]) * std::atan(0.5 * avail / eps));
        if (wsec > 0.5 * avail) wsec = 0.5 * avail;
        if (wsec < 0.0) wsec = 0.0;
        enew = avail - wsec;
        T.energy[ORC_OE_LOSS_IONIZ] += ion_e;
        const double cp = avail > 0.0 ? std::sqrt(enew / avail) : 1.0;
        const double sp = avail > 0.0 ? std::sqrt(wsec / avail) : 0.0;
        double nd[3], sd[3];
        turn(dir, cp, cph, sph, nd);
        turn(dir, sp, -cph, -sph, sd);            /* secondary azimuth = primary azimuth - pi */
        set_u(P, enew, nd);
        OParticle S;
        for (int i = 0; i < 3; ++i) S.x[i] = P.x[i];
        S.species = SP_E; S.node = child_node(P.node, ev_coll, 0);
        S.t_alive = 0.0; S.ev = 0;
        set_u(S, wsec, sd);
        T.ledger[ORC_OB_BIRTHS + SP_E] += 1;
        T.ledger[ORC_OB_N_SPAWN_E] += 1;
        if (wsec < p->e_cut_ev) die(S, ORC_OR_CUTOFF, ORC_OE_CUTOFF, wsec);
        else stack.push_back(S);
        const int ion = p->species_out[ch];
        if (ion >= 0) {
          OParticle I;
          for (int i = 0; i < 3; ++i) I.x[i] = P.x[i];
          I.species = ion; I.node = child_node(P.node, ev_coll, 1);
          I.t_alive = 0.0; I.ev = 0;
          double ei, di[3];
          thermal3(0, I.node, DOM_ION_BIRTH, &ei, di);
          set_u(I, ei, di);
          T.energy[ORC_OE_IN_THERMAL] += ei;
          T.ledger[ORC_OB_BIRTHS + ion] += 1;
          T.ledger[ORC_OB_N_SPAWN_ION] += 1;
          stack.push_back(I);
        }
      } else {                                   /* clustering: the product replaces the ion */
        write_end(es, P);
        die(P, ORC_OR_CLUSTER, ORC_OE_CLUSTER, ec);
        OParticle C;
        for (int i = 0; i < 3; ++i) C.x[i] = P.x[i];
        C.species = p->species_out[ch];
        C.node = child_node(P.node, ev_coll, 2);
        C.t_alive = 0.0; C.ev = 0;
        double ecl, dc[3];
        thermal3(ev_coll, P.node, DOM_CLUSTER, &ecl, dc);
        set_u(C, ecl, dc);
        T.energy[ORC_OE_IN_THERMAL] += ecl;
        T.ledger[ORC_OB_BIRTHS + C.species] += 1;
        P = C;
        continue;
      }
      /* ---- terminator (Sec. 3.2) ---- */
      if (s == SP_E && enew < p->e_cut_ev) {
        write_end(es, P); die(P, ORC_OR_CUTOFF, ORC_OE_CUTOFF, enew); return;
      }
      if (P.ev >= p->max_collisions) {
        write_end(es, P); die(P, ORC_OR_CAP_COLL, ORC_OE_CAP, enew); return;
      }
      if (P.t_alive >= p->max_lifetime_s) {
        write_end(es, P); die(P, ORC_OR_CAP_TIME, ORC_OE_CAP, enew); return;
      }
    }
  }

  void run_range(const orc_orbit_primaries* pr, int64_t lo, int64_t hi, uint64_t* per_primary,
                 double* end_state) {
    const orc_problem* p = R->p;
    std::vector<OParticle> stack;
    for (int64_t i = lo; i < hi; ++i) {
      pid = (uint64_t)(pr->pid_offset + i);
      tree_collisions = 0;
      OParticle P;
      P.x[0] = pr->x_m[i]; P.x[1] = pr->y_m[i]; P.x[2] = pr->z_m[i];
      P.species = pr->species[i];
      P.node = 0; P.t_alive = 0.0; P.ev = 0;
      const double mu = pr->mu[i];
      const double st = std::sqrt(std::fmax(0.0, 1.0 - mu * mu));
      const double d[3] = {st * std::cos(pr->phi[i]), st * std::sin(pr->phi[i]), mu};
      set_u(P, pr->e_ev[i], d);
      double* es = end_state ? end_state + 8 * i : nullptr;
      T.energy[ORC_OE_IN_PRIMARY] += pr->e_ev[i];
      T.ledger[ORC_OB_BIRTHS + P.species] += 1;
      if (P.species == SP_E && pr->e_ev[i] < p->e_cut_ev) {
        write_end(es, P);
        die(P, ORC_OR_CUTOFF, ORC_OE_CUTOFF, pr->e_ev[i]);
      } else {
        stack.push_back(P);
      }
      while (!stack.empty()) {
        OParticle Q = stack.back();
        stack.pop_back();
        transport(Q, stack, Q.node == 0 ? es : nullptr);
      }
      if (per_primary) per_primary[i] += tree_collisions;
    }
  }
};

int check_orbit(const orc_problem* p, const orc_orbit* o, const orc_orbit_primaries* pr) {
  if (check_problem(p) || !o || !pr || !(o->tube_radius_m > 0.0) || o->n_rbins < 1) return 1;
  for (int s = 0; s < ORC_N_SPECIES; ++s)
    if (!(o->dt_s[s] > 0.0)) return 1;
  for (int k = 0; k < p->n_channels; ++k) {
    const int kd = p->kind[k];
    if (kd == RECOMBINATION || kd == CHARGE_EXCHANGE) return 2;
    if ((kd == ELASTIC || kd == IONIZATION) && p->target && p->target[k] != 0) return 2;
  }
  const double R2 = o->tube_radius_m * o->tube_radius_m;
  for (int64_t i = 0; i < pr->n; ++i) {
    const double x = pr->x_m[i], y = pr->y_m[i], z = pr->z_m[i];
    if (!(x * x + y * y < R2) || !(z >= 0.0 && z <= p->length_m) || pr->species[i] >= ORC_N_SPECIES)
      return 3;
  }
  return 0;
}

}  // namespace

extern "C" {

void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  philox4x64_10(ctr, key, out);
}

double orc_sigma(const orc_problem* p, int channel, double e_ev) { return sigma_at(p, channel, e_ev); }

double orc_sample_angle(const orc_problem* p, int channel, double e_ev, double u) {
  return sample_angle(p, channel, e_ev, u);
}

void orc_elastic_moving_target(const orc_problem* p, double m1_ev, double e_ev, double mu,
                               const uint64_t w[4], const uint64_t ctr[3], const uint64_t key[2],
                               double* out_e, double* out_mu, double* v) {
  struct Ctx { const uint64_t* ctr; const uint64_t* key; } cx = {ctr, key};
  auto blk = [](void* c, uint64_t k, uint64_t out[4]) {
    Ctx* q = (Ctx*)c;
    const uint64_t full[4] = {q->ctr[0], q->ctr[1], q->ctr[2], k};
    philox4x64_10(full, q->key, out);
  };
  int ch = 0;
  for (int k = 0; k < p->n_channels; ++k)
    if (p->kind[k] == ELASTIC) { ch = k; break; }
  moving_target_elastic(p, ch, m1_ev, e_ev, mu, w, blk, &cx, out_e, out_mu, v);
}

void orc_ionization_moving_target(const orc_problem* p, int channel, double m1_ev, double e_ev,
                                  double mu, double m_ion_ev, const uint64_t w[4],
                                  const uint64_t ctr[3], const uint64_t key[2], double out[7]) {
  struct Ctx { uint64_t ctr[3]; uint64_t key[2]; } cx = {{ctr[0], ctr[1], ctr[2]}, {key[0], key[1]}};
  auto blk = [](void* c, uint64_t k, uint64_t o4[4]) {
    Ctx* q = (Ctx*)c;
    const uint64_t full[4] = {q->ctr[0], q->ctr[1], q->ctr[2], k};
    philox4x64_10(full, q->key, o4);
  };
  IonOut io;
  moving_target_ionization(p, channel, m1_ev, e_ev, mu, m_ion_ev, w, blk, &cx, &io);
  out[0] = io.e1; out[1] = io.mu1; out[2] = io.e2; out[3] = io.mu2;
  out[4] = io.eion; out[5] = io.muion; out[6] = io.ei;
}

void orc_charge_exchange(const orc_problem* p, double m1_ev, double e_ev, double mu,
                         const uint64_t ctr[3], const uint64_t key[2], double* out_e,
                         double* out_mu, double* v2) {
  struct Ctx { uint64_t ctr[3]; uint64_t key[2]; } cx = {{ctr[0], ctr[1], ctr[2]}, {key[0], key[1]}};
  auto blk = [](void* c, uint64_t k, uint64_t out[4]) {
    Ctx* q = (Ctx*)c;
    const uint64_t full[4] = {q->ctr[0], q->ctr[1], q->ctr[2], k};
    philox4x64_10(full, q->key, out);
  };
  double v[3];
  charge_exchange(p, m1_ev, e_ev, mu, blk, &cx, out_e, out_mu, v);
  if (v2) for (int i = 0; i < 3; ++i) v2[i] = v[i];
}

int orc_collide(const orc_problem* p, int ch, int species, double e_ev, double mu,
                const uint64_t w[4], double* out_e, double* out_mu, int* out_species) {
  /* same kinematics as Worker::transport, for single-collision enumeration */
  double m = p->species_mass_ev[species];
  int64_t eq = quant_e(e_ev);
  double e = (double)eq / Q_ENERGY;
  int kind = p->kind[ch];
  if (kind == ELASTIC) {
    double g = m / p->target_mass_ev;
    double cchi = sample_angle(p, ch, e, u01(w[2]));
    double a = 1.0 + 2.0 * g * cchi + g * g;
    double ct = (cchi + g) / std::sqrt(a);
    int64_t rq = quant_recoil(e * 2.0 * g * (1.0 - cchi) / ((1.0 + g) * (1.0 + g)));
    if (rq > eq) rq = eq;
    int64_t eq1 = eq - rq;
    double st = std::sqrt(std::fmax(0.0, 1.0 - ct * ct));
    double cphi = std::cos(TWO_PI * u01(w[3]));
    double smu = std::sqrt(std::fmax(0.0, 1.0 - mu * mu));
    out_e[0] = (double)eq1 / Q_ENERGY;
    out_mu[0] = std::fmax(-1.0, std::fmin(1.0, mu * ct + smu * st * cphi));
    out_species[0] = species;
    return 1;
  }
  if (kind == EXCITATION) {
    out_e[0] = (double)(eq - quant_e(p->loss_ev[ch])) / Q_ENERGY;
    out_mu[0] = mu; out_species[0] = species;
    return 1;
  }
  if (kind == IONIZATION) {
    int64_t iq = quant_e(p->loss_ev[ch]);
    int64_t avail = eq - iq;
    double eps = p->ioniz_eps_ev;
    double wmax = (e - p->loss_ev[ch]) * 0.5;
    double wsec = eps * std::tan(u01(w[2]) * std::atan(wmax / eps));
    int64_t wq = quant_e(wsec);
    if (wq > avail / 2) wq = avail / 2;
    if (wq < 0) wq = 0;
    int64_t eq1 = avail - wq;
    double c2p = avail > 0 ? (double)eq1 / (double)avail : 1.0;
    double c2s = avail > 0 ? (double)wq / (double)avail : 0.0;
    double cp = std::sqrt(c2p), sp = std::sqrt(c2s);
    double cphi = std::cos(TWO_PI * u01(w[3]));
    double smu = std::sqrt(std::fmax(0.0, 1.0 - mu * mu));
    out_e[0] = (double)eq1 / Q_ENERGY;
    out_mu[0] = std::fmax(-1.0, std::fmin(1.0, mu * cp + smu * sp * cphi));
    out_species[0] = species;
    out_e[1] = (double)wq / Q_ENERGY;
    out_mu[1] = std::fmax(-1.0, std::fmin(1.0, mu * sp - smu * cp * cphi));
    out_species[1] = SP_E;
    return 2;
  }
  if (kind == CLUSTERING || kind == CLUSTERING3) {
    double kt = KB_EV * p->gas_temperature_k;
    double c = std::cos(TWO_PI * u01(w[2]));
    double ec = kt * (-std::log(eta01(w[0])) - std::log(eta01(w[1])) * c * c);
    out_e[0] = (double)quant_e(ec) / Q_ENERGY;
    out_mu[0] = 2.0 * u01(w[3]) - 1.0;
    out_species[0] = p->species_out[ch];
    return 1;
  }
  return 0;   /* recombination: no products */
}

int orc_run_pass(const orc_problem* p, const orc_primaries* pr, uint64_t seed, int pass,
                 const uint64_t* field_time_in, int mode, int n_threads, orc_tallies* out) {
  if (check_problem(p) || !pr || !out || (pass != 1 && pass != 2)) return 1;
  return do_pass(p, pr, seed, pass, field_time_in, nullptr, (double)pr->n_decays, false, mode,
                 n_threads, out);
}

int orc_run_cycle(const orc_problem* p, const orc_primaries* pr, uint64_t seed,
                  const uint64_t* field_time_in, const uint64_t* field_recomb_in,
                  double field_decays, int mode, int n_threads, orc_tallies* out) {
  if (check_problem(p) || !pr || !out) return 1;
  if (field_time_in && !(field_decays > 0.0)) return 1;
  return do_pass(p, pr, seed, 2, field_time_in, field_recomb_in, field_decays, !field_time_in,
                 mode, n_threads, out);
}

int orc_run(const orc_problem* p, const orc_primaries* pr, uint64_t seed, int n_passes,
            int mode, int n_threads, orc_tallies* out) {
  if (check_problem(p) || !pr || !out || n_passes < 1 || n_passes > 2) return 1;
  int nz = p->n_zbins, ntb = p->n_tebins;
  size_t ntime = (size_t)ORC_N_SPECIES * (nz + 2) * ntb;
  /* pass 1 into out; if two passes, keep its time tally and rerun */
  int rc = do_pass(p, pr, seed, 1, nullptr, nullptr, 0.0, false, mode, n_threads, out);
  if (rc) return rc;
  std::vector<uint64_t> time1(out->time_fx, out->time_fx + ntime);
  if (n_passes == 2) {
    /* the run's counts of both passes survive the reset of the pass-1 tallies */
    const int64_t coll1 = out->ledger[ORC_N_COLLISIONS_ALL];
    const int64_t flights1 = out->ledger[ORC_N_FLIGHTS_ALL];
    std::memset(out->spectrum, 0, sizeof(uint64_t) * 2 * ORC_N_SPECIES * (p->n_spec_bins + 1));
    std::memset(out->time_fx, 0, sizeof(uint64_t) * ntime);
    std::memset(out->cross_pos, 0, sizeof(uint64_t) * ORC_N_SPECIES * (nz + 1));
    std::memset(out->cross_neg, 0, sizeof(uint64_t) * ORC_N_SPECIES * (nz + 1));
    std::memset(out->recomb, 0, sizeof(uint64_t) * ORC_N_SPECIES * nz);
    std::memset(out->ledger, 0, sizeof(int64_t) * ORC_LEDGER_LEN);
    std::memset(out->chan_count, 0, sizeof(uint64_t) * p->n_channels);
    if (out->per_primary) std::memset(out->per_primary, 0, sizeof(uint64_t) * pr->n);
    rc = do_pass(p, pr, seed, 2, time1.data(), nullptr, (double)pr->n_decays, false, mode,
                 n_threads, out);
    if (rc) return rc;
    out->ledger[ORC_N_COLLISIONS_ALL] += coll1;
    out->ledger[ORC_N_FLIGHTS_ALL] += flights1;
  }
  /* normalisation: Eq. target_field_density, current j = (N+ - N-)/(A t_sim) */
  double dz = p->length_m / nz;
  double tsim = (double)pr->n_decays / p->activity_bq;
  double vol = dz * p->area_m2;
  for (int s = 0; s < ORC_N_SPECIES; ++s) {
    for (int j = 0; j < nz; ++j) {
      double tsum = 0.0, t1 = 0.0;
      for (int b = 0; b < ntb; ++b) {
        size_t idx = ((size_t)s * (nz + 2) + (j + 1)) * ntb + b;
        tsum += (double)out->time_fx[idx] / Q_TIME;
        double nb = (double)time1[idx] / Q_TIME / (tsim * vol);
        t1 += nb;
        if (out->field) out->field[((size_t)s * nz + j) * ntb + b] = nb;
      }
      if (out->density)
        out->density[(size_t)s * nz + j] =
            tsum / (tsim * vol) - (double)out->recomb[(size_t)s * nz + j] / vol;
      (void)t1;
    }
    if (out->current)
      for (int k = 0; k <= nz; ++k) {
        size_t idx = (size_t)s * (nz + 1) + k;
        out->current[idx] =
            ((double)out->cross_pos[idx] - (double)out->cross_neg[idx]) / (p->area_m2 * tsim);
      }
  }
  return 0;
}


int orc_orbit_run(const orc_problem* p, const orc_orbit* o, const orc_orbit_primaries* pr,
                  uint64_t seed, int n_threads, orc_orbit_tallies* out) {
  const int bad = check_orbit(p, o, pr);
  if (bad) return bad;
  if (!out) return 1;
  OrbitRun R;
  R.p = p; R.o = o; R.seed = seed;
  R.dz = p->length_m / p->n_zbins;
  R.inv_dz = (double)p->n_zbins / p->length_m;
  R.r_scale = (double)o->n_rbins / o->tube_radius_m;
  R.edge2.resize((size_t)o->n_rbins + 1);
  for (int k = 0; k <= o->n_rbins; ++k) {
    const double rk = o->tube_radius_m * (double)k / (double)o->n_rbins;
    R.edge2[k] = rk * rk;
  }
  R.fields = o->e_r_vm2 != 0.0;
  if (o->e_z_vm)
    for (int j = 0; j < p->n_zbins; ++j) R.fields = R.fields || o->e_z_vm[j] != 0.0;
  R.max_steps = o->max_steps ? o->max_steps : (1ULL << 40);
  if (n_threads < 1) n_threads = 1;
  if ((int64_t)n_threads > pr->n) n_threads = (int)(pr->n > 0 ? pr->n : 1);
  std::vector<OWorker> W(n_threads);
  std::vector<std::thread> th;
  for (int t = 0; t < n_threads; ++t) {
    W[t].R = &R;
    W[t].T.init(p, o);
    int64_t lo = pr->n * t / n_threads, hi = pr->n * (t + 1) / n_threads;
    auto job = [&W, t, pr, lo, hi, out] { W[t].run_range(pr, lo, hi, out->per_primary, out->end_state); };
    if (n_threads == 1) job();
    else th.emplace_back(job);
  }
  for (auto& x : th) x.join();
  for (int t = 0; t < n_threads; ++t) {
    const OTally& T = W[t].T;
    auto add = [](uint64_t* dst, const std::vector<uint64_t>& src) {
      for (size_t i = 0; i < src.size(); ++i) dst[i] += src[i];
    };
    add(out->spectrum, T.spectrum); add(out->time_z, T.time_z); add(out->time_r, T.time_r);
    add(out->cross_pos, T.cross_pos); add(out->cross_neg, T.cross_neg);
    add(out->rcross_out, T.rcross_out); add(out->rcross_in, T.rcross_in);
    add(out->wall, T.wall); add(out->chan_count, T.chan_count);
    for (int i = 0; i < ORC_OB_LEDGER_LEN; ++i) out->ledger[i] += T.ledger[i];
    for (int i = 0; i < ORC_OE_LEN; ++i) out->energy[i] += T.energy[i];
  }
  return 0;
}

}  /* extern "C" */
