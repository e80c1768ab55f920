// transport.cu - persistent Monte Carlo transport kernel of the KARL hot path.
//
// One launch runs one pass over all primaries of a run (Sec. 2.1 main cycle,
// Fig. 1).  Every lane holds one particle in registers and performs one event
// per loop iteration: a free flight by optical depth (Eqs. mean_free_path and
// distance_from_mfp over the piecewise-constant column, equal in law to the
// segment-stop mover of Sec. 3.1), the time/density and current tallies of
// Secs. 2.2-2.3 as range adds, the terminator of Sec. 3.2, a channel chosen
// with probability sigma_i n_i / sum_j sigma_j n_j, and its kinematics
// (Sec. 3.3).  Products go to a device-wide ring; lanes whose particle ended
// take the next one from the ring (products first) or from the primaries.
// All waits are bounded by iteration counts and a wall-clock deadline, after
// which the kernel records an error and returns.
#include "karl_device.cuh"

namespace karl {

constexpr double Q_E = 16777216.0;             // 2^24 energy units per eV
constexpr double INV_Q_E = 1.0 / 16777216.0;
constexpr double Q_T = 1125899906842624.0;     // 2^50 time units per s
constexpr double C_LIGHT = 299792458.0;
constexpr unsigned FULL = 0xffffffffu;
constexpr long long SPIN_LIMIT = 1LL << 26;    // bounded waits on ring cells

template <bool F32> struct RT;
template <> struct RT<false> {
  using R = double;
  static __device__ __forceinline__ R u(unsigned long long w) { return u01d(w); }
  static __device__ __forceinline__ R eta(unsigned long long w) { return eta01d(w); }
  static __device__ __forceinline__ R lg(R x) { return log(x); }
  static __device__ __forceinline__ R sq(R x) { return sqrt(x); }
  static __device__ __forceinline__ R rsq(R x) { return rsqrt(x); }
  static __device__ __forceinline__ R tn(R x) { return tan(x); }
  static __device__ __forceinline__ R atn(R x) { return atan(x); }
  static __device__ __forceinline__ R cpi(R x) { return cospi(x); }
  static __device__ __forceinline__ R tab(const Params& P, int k, int i) {
    return __ldg(P.sig + (size_t)i * P.nch + k);      // [node][channel]
  }
  static __device__ __forceinline__ R energy(long long eq) { return (double)eq * (1.0 / 16777216.0); }
  static __device__ __forceinline__ long long quant_de(R de) {
    return (long long)floor(de * 16777216.0 + 0.5);
  }
};
template <> struct RT<true> {
  using R = float;
  static __device__ __forceinline__ R u(unsigned long long w) { return u01f(w); }
  static __device__ __forceinline__ R eta(unsigned long long w) { return eta01f(w); }
  static __device__ __forceinline__ R lg(R x) { return logf(x); }
  static __device__ __forceinline__ R sq(R x) { return sqrtf(x); }
  static __device__ __forceinline__ R rsq(R x) { return rsqrtf(x); }
  static __device__ __forceinline__ R tn(R x) { return tanf(x); }
  static __device__ __forceinline__ R atn(R x) { return atanf(x); }
  static __device__ __forceinline__ R cpi(R x) { return cospif(x); }
  static __device__ __forceinline__ R tab(const Params& P, int k, int i) {
    return __ldg(P.sigf + (size_t)i * P.nch + k);     // [node][channel]
  }
  // energy from 2^-24 eV units with 32-bit conversions (below 65 keV)
  static __device__ __forceinline__ R energy(long long eq) {
    return eq < (1LL << 40) ? (float)(unsigned)(eq >> 8) * (1.0f / 65536.0f)
                            : (float)eq * (1.0f / 16777216.0f);
  }
  static __device__ __forceinline__ long long quant_de(R de) {
    const float x = de * 16777216.0f + 0.5f;
    return x < 2.0e9f ? (long long)__float2int_rz(x) : (long long)x;
  }
};

struct Lane {
  double z;
  long long eq;                 // kinetic energy, 2^-24 eV
  double mu;                    // pitch cosine
  unsigned long long node;      // lineage id
  double tal;                   // time alive (tracked only under a lifetime cap)
  unsigned long long pid;       // primary id
  unsigned ev;                  // collisions so far = index of the next flight
  int sp;                       // species
  int j;                        // segment holding z (carried from the last flight)
};

__device__ __forceinline__ double face(const Params& P, int k) {
  return k >= P.nz ? P.L : (double)k * P.dz;
}
__device__ __forceinline__ int segment_of(const Params& P, double z) {
  int j = (int)floor(z / P.dz);
  return j < 0 ? 0 : (j > P.nz - 1 ? P.nz - 1 : j);
}
__device__ __forceinline__ unsigned long long quant_t(double len, double inv_sz) {
  double t = len * inv_sz;
  return (unsigned long long)(t * Q_T + 0.5);
}
__device__ __forceinline__ long long quant_e(double e) { return (long long)floor(e * Q_E); }

template <class R>
__device__ __forceinline__ R speed(R e, R inv_m) {
  R x = e * inv_m;
  return (R)C_LIGHT * sqrt(x * ((R)2 + x)) / ((R)1 + x);
}

struct Shared {
  unsigned long long ledger[LEDGER];
  unsigned long long chan[MAXCH];
};

__device__ __forceinline__ void sadd(unsigned long long* p, long long v) {
  atomicAdd(p, (unsigned long long)v);
}

// Range add of q over rows [a, b] (inclusive) of a difference array with row
// stride `stride`; rows are then recovered by a prefix sum.
__device__ __forceinline__ void range_add(unsigned long long* d, int a, int b, size_t stride,
                                          unsigned long long q) {
  if (a > b) return;
  atomicAdd(d + (size_t)a * stride, q);
  atomicAdd(d + (size_t)(b + 1) * stride, (unsigned long long)0 - q);
}

// ---------------------------------------------------------------------------
// ring cells

__device__ bool ring_put(const Ring& R, Control* ctl, unsigned long long pos, const Lane& p,
                         unsigned long long deadline) {
  unsigned long long* cell = R.seq + (pos & R.mask);
  long long spins = 0;
  while (ld_acquire(cell) != pos) {           // previous occupant not consumed yet
    if (++spins > SPIN_LIMIT || ((spins & 1023) == 0 && globaltimer_ns() > deadline)) {
      atomicCAS(&ctl->error, 0, ERR_CAPACITY);
      atomicExch(&ctl->abort, 1);
      return false;
    }
    __nanosleep(64);
  }
  size_t i = pos & R.mask;
  R.z[i] = p.z; R.eq[i] = p.eq; R.mu[i] = p.mu; R.node[i] = p.node; R.tal[i] = p.tal;
  R.pid[i] = p.pid; R.ev[i] = p.ev; R.sj[i] = ((unsigned)p.j << 8) | (unsigned)p.sp;
  st_release(cell, pos + 1);
  return true;
}

__device__ bool ring_get(const Ring& R, Control* ctl, unsigned long long pos, Lane& p,
                         unsigned long long deadline) {
  unsigned long long* cell = R.seq + (pos & R.mask);
  long long spins = 0;
  while (ld_acquire(cell) != pos + 1) {        // producer still writing
    if (++spins > SPIN_LIMIT || ((spins & 1023) == 0 && globaltimer_ns() > deadline)) {
      atomicCAS(&ctl->error, 0, ERR_TIMEOUT);
      atomicExch(&ctl->abort, 1);
      return false;
    }
    __nanosleep(32);
  }
  size_t i = pos & R.mask;
  p.z = R.z[i]; p.eq = R.eq[i]; p.mu = R.mu[i]; p.node = R.node[i]; p.tal = R.tal[i];
  p.pid = R.pid[i]; p.ev = R.ev[i];
  const unsigned sj = R.sj[i];
  p.sp = (int)(sj & 0xffu);
  p.j = (int)(sj >> 8);
  st_release(cell, pos + R.cap);
  return true;
}

// ---------------------------------------------------------------------------
// one event of one particle

struct EventOut {
  bool alive;
  int chan;                               // channel of this event's collision, -1 if none
  unsigned long long flights, colls;      // per-lane counters, flushed at the end
  unsigned long long recoil, excit;       // per-lane energy sums (2^-24 eV)
};

// Products of a warp's events go to a short last-in-first-out queue in the
// warp's shared memory and are taken by the warp's idle lanes, so a primary's
// products are followed close to depth first (the paper follows a particle
// list).  The queue spills to the shared ring when full, and once the
// primaries are used up, so idle warps elsewhere can share the last work.
constexpr int WQ = 32;
constexpr int WARPS = 8;                  // 256-thread blocks
struct WarpQueue {
  Lane s[WQ];
  int top;
};

struct RingPort {
  const Ring* R;
  Control* ctl;
  unsigned long long deadline;
  WarpQueue* q;
  bool local;              // primaries remain: keep products in the warp queue
  unsigned long long spilled;
};

__device__ __forceinline__ void emit(RingPort& port, const Lane& p) {
  if (port.local) {
    const int i = atomicAdd(&port.q->top, 1);
    if (i < WQ) {
      port.q->s[i] = p;
      atomicAdd((unsigned long long*)&port.ctl->active, 1ULL);   // held by this warp
      return;
    }
  }
  unsigned long long pos = atomicAdd(&port.ctl->tail, 1ULL);
  ring_put(*port.R, port.ctl, pos, p, port.deadline);
  port.spilled += 1;
}

template <bool F32>
__device__ __forceinline__ void die(const Params& P, Shared& S, Lane& L, int reason, int slot) {
  sadd(&S.ledger[L_DEATHS + L.sp * NREASON + reason], 1);
  sadd(&S.ledger[slot], L.eq);
  if (P.per_primary) atomicAdd(P.per_primary + (L.pid - (unsigned long long)P.pid_offset),
                               (unsigned long long)L.ev);
}

template <bool F32>
__device__ __forceinline__ void thermal(const Params& P, const unsigned long long w[4],
                                        long long& eq, double& mu) {
  // Maxwell-Boltzmann target: Gamma(3/2, kT) = Exp(1) + Z^2/2 (Box-Muller), isotropic
  double c = cospi(2.0 * u01d(w[2]));
  double e = P.kT * (-log(eta01d(w[0])) - log(eta01d(w[1])) * c * c);
  eq = quant_e(e);
  mu = 2.0 * u01d(w[3]) - 1.0;
}

template <bool F32>
__device__ void event(const Params& P, Shared& S, Lane& L, EventOut& o, RingPort& port) {
  using T = RT<F32>;
  using R = typename T::R;
  o.alive = true;
  o.chan = -1;
  if (L.eq <= 0) {                 // no kinetic energy: the particle never moves
    die<F32>(P, S, L, R_STALLED, L_E_STALLED);
    o.alive = false;
    return;
  }
  const int s = L.sp;
  const R e = T::energy(L.eq);
  const R v = speed<R>(e, (R)P.inv_mass[s]);

  unsigned long long w[4];
  philox4x64_10((unsigned long long)L.ev, L.node,
                ((unsigned long long)P.pass << 8) | DOM_EVENT, 0ULL, P.seed, L.pid, w);
  const R tau = -T::lg(T::eta(w[0]));
  o.flights += 1;

  // per-flight coefficients: sigma_k(E) (gas, electron recombination) or 1/v
  // (ion recombining with the electron field, whose rate already has sigma v)
  const int nsc = P.nsc[s];
  R coef[MAXSPCH];
  const R le = T::lg(e * (R)P.inv_e_min);       // ln(E / e_min), shared by both lookups
  const R lx = le * (R)P.inv_h;
  int ti = (int)floor(lx);
  R tf;
  if (ti < 0) { ti = 0; tf = (R)0; }
  else if (ti > P.n_energy - 2) { ti = P.n_energy - 2; tf = (R)1; }
  else { tf = lx - (R)ti; }
  R gas = (R)0;
  int nrec = 0;
  double rc0 = 0.0, rc1 = 0.0;
  const double* rcol0 = P.colgas;
  const double* rcol1 = P.colgas;
  const double* rrate0 = P.nseg;
  const double* rrate1 = P.nseg;
#pragma unroll
  for (int c = 0; c < MAXSPCH; ++c) {
    if (c >= nsc) break;
    const int k = P.sc[s][c];
    const ChanDev& ch = P.ch[k];
    R cv;
    if (ch.kind == RECOMBINATION && s != SP_E) {
      cv = (R)1 / v;
    } else if (L.eq > ch.thr_q) {
      const R a0 = T::tab(P, k, ti);
      cv = a0 + tf * (T::tab(P, k, ti + 1) - a0);
    } else {
      cv = (R)0;
    }
    coef[c] = cv;
    if (ch.kind != RECOMBINATION) {
      gas += cv;
    } else {
      if (nrec == 0) { rc0 = (double)cv; rcol0 = P.fcol[k]; rrate0 = P.frate[k]; }
      else { rc1 = (double)cv; rcol1 = P.fcol[k]; rrate1 = P.frate[k]; }
      ++nrec;
    }
  }
  // energy bin of the time tally
  int b = 0;
  if (P.ntb > 1) {
    b = (int)floor(le * (R)P.tb_scale);
    b = b < 0 ? 0 : (b > P.ntb - 1 ? P.ntb - 1 : b);
  }
  const size_t trow = (size_t)P.ntb;                         // stride between z rows
  const size_t tbase = (size_t)s * (P.nz + 2) * P.ntb + b;   // (s, row 0, b)
  const size_t xbase = (size_t)s * (P.nz + 2);
  const double gasd = (double)gas;

  // G(k) = optical-depth column of the whole rate to face k, and the rate in
  // segment j (the column tables may live in shared memory: plain loads)
  auto colsum = [&](int k) -> double {
    double g = gasd * P.colgas[k];
    if (nrec > 0) g += rc0 * rcol0[k];
    if (nrec > 1) g += rc1 * rcol1[k];
    return g;
  };
  auto segrate = [&](int j) -> double {
    double r = gasd * P.nseg[j];
    if (nrec > 0) r += rc0 * rrate0[j];
    if (nrec > 1) r += rc1 * rrate1[j];
    return r;
  };

  const int j0 = L.j;
  double zc;
  int jc;
  int exit_end = -1;
  double inv_sz = 0.0;
  if (L.mu == 0.0) {
    // no motion along z: collide in place after path tau / rate
    jc = j0;
    const double r = segrate(jc);
    if (!(r > 0.0)) {
      die<F32>(P, S, L, R_STALLED, L_E_STALLED);
      o.alive = false;
      return;
    }
    const double tfl = (double)tau / r / (double)v;
    atomicAdd(P.time_pt + tbase + (size_t)(jc + 1) * trow, (unsigned long long)(tfl * Q_T + 0.5));
    if (P.track_time) L.tal += tfl;
    zc = L.z;
  } else {
    // One code path for both directions: the flight ends where the column of
    // the rate, G, reaches G(z0) +- tau |mu| (optical depth along the path).
    const bool up = L.mu > 0.0;
    const double amu = fabs(L.mu);
    const int nz = P.nz;
    const double g0 = colsum(j0) + segrate(j0) * (L.z - P.faces[j0]);
    const double delta = (double)tau * amu;
    const double target = up ? g0 + delta : g0 - delta;
    const bool ex = up ? !(target < colsum(nz)) : !(target > 0.0);
    if (ex) {
      exit_end = up ? 1 : 0;
      zc = up ? P.L : 0.0;
      jc = up ? nz - 1 : 0;
    } else {
      // largest k with G(k) <= target, in [j0, nz) going up, [0, j0] going down
      int lo = up ? j0 : 0, hi = up ? nz : j0 + 1;
      if (nrec == 0 && gasd > 0.0 && P.nq > 0) {
        // bracket from the inverse gas-column table (exact with gas only)
        const double q = target / gasd * P.nq_over_colmax;
        if (q >= 0.0 && q < (double)P.nq) {
          const int qi = (int)q;
          const int a = max(lo, P.ginv[qi] - 1), bb = min(hi, P.ginv[qi + 1] + 1);
          if (a < bb && colsum(a) <= target && target < colsum(bb)) { lo = a; hi = bb; }
        }
      }
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (colsum(mid) <= target) lo = mid; else hi = mid;
      }
      jc = lo;
      const double fj = P.faces[jc], fj1 = P.faces[jc + 1];
      const double gap = target - colsum(jc);
      const double r = segrate(jc);
      if (F32) zc = fj + (double)((float)gap / (float)r);
      else zc = fj + gap / r;
      zc = fmin(fmax(zc, fj), fj1);
      zc = up ? fmax(zc, L.z) : fmin(zc, L.z);
    }
    // time in each segment crossed (Sec. 2.2) as point adds at both ends and
    // one range add of the full-segment time, and the face crossings (Sec. 2.3)
    inv_sz = 1.0 / (amu * (double)v);
    const size_t row0 = tbase + (size_t)(j0 + 1) * trow;
    if (jc == j0) {
      atomicAdd(P.time_pt + row0, quant_t(fabs(zc - L.z), inv_sz));
    } else {
      const double fs = P.faces[up ? j0 + 1 : j0];
      atomicAdd(P.time_pt + row0, quant_t(fabs(fs - L.z), inv_sz));
      const unsigned long long qf = quant_t(P.dz, inv_sz);
      const double fe = P.faces[up ? jc : jc + 1];
      atomicAdd(P.time_pt + tbase + (size_t)(jc + 1) * trow, ex ? qf : quant_t(fabs(zc - fe), inv_sz));
      const int lo_seg = min(j0, jc), hi_seg = max(j0, jc);
      range_add(P.time_rg + tbase, lo_seg + 2, hi_seg, trow, qf);   // full segments
    }
    const int fa = up ? j0 + 1 : (ex ? 0 : jc + 1);
    const int fb = up ? (ex ? nz : jc) : j0;
    range_add((up ? P.xpos_rg : P.xneg_rg) + xbase, fa, fb, 1, 1ULL);
    if (P.track_time) L.tal += fabs(zc - L.z) * inv_sz;
  }
  if (exit_end >= 0) {
    long long bin = L.eq / P.spec_bin_q;
    if (bin > P.nspec) bin = P.nspec;
    atomicAdd(P.spectrum + ((size_t)exit_end * NSP + s) * (P.nspec + 1) + bin, 1ULL);
    die<F32>(P, S, L, exit_end == 0 ? R_EXIT0 : R_EXIT1, exit_end == 0 ? L_E_EXIT0 : L_E_EXIT1);
    o.alive = false;
    return;
  }
  L.z = zc;
  L.j = jc;

  // ---- collision in segment jc: channel with probability rate_k / rate_tot ----
  L.ev += 1;
  o.colls += 1;
  int chs = -1, last = -1;
  if (nrec == 0) {
    // gas channels only: the density of segment jc factors out
    const R target = T::u(w[1]) * gas;
    R cum = (R)0;
#pragma unroll
    for (int c = 0; c < MAXSPCH; ++c) {
      if (c >= nsc) break;
      if (!(coef[c] > (R)0)) continue;
      last = c;
      cum += coef[c];
      if (target < cum) { chs = c; break; }
    }
  } else {
    const double nj = P.nseg[jc];
    const double target = u01d(w[1]) * segrate(jc);
    double cum = 0.0;
#pragma unroll
    for (int c = 0; c < MAXSPCH; ++c) {
      if (c >= nsc) break;
      const int kk = P.sc[s][c];
      const double rk = (double)coef[c] * (P.ch[kk].kind == RECOMBINATION ? P.frate[kk][jc] : nj);
      if (!(rk > 0.0)) continue;
      last = c;
      cum += rk;
      if (target < cum) { chs = c; break; }
    }
  }
  if (chs < 0) chs = last;
  const int k = P.sc[s][chs];
  o.chan = k;
  const ChanDev ch = P.ch[k];
  if (ch.kind == ELASTIC) {
    // isotropic in CM, target at rest: lab polar angle and energy transfer
    const R g = (R)P.gam[s];
    const R cchi = (R)2 * T::u(w[2]) - (R)1;
    const R a = (R)1 + (R)2 * g * cchi + g * g;
    const R ct = (cchi + g) * T::rsq(a);
    // energy given to the target, E - E' = E 2g(1 - cos chi)/(1+g)^2
    const R de = e * ((R)2 * g) * ((R)1 - cchi) * (R)P.inv_1pg2[s];
    long long rq = T::quant_de(de);
    if (rq > L.eq) rq = L.eq;
    o.recoil += (unsigned long long)rq;
    L.eq -= rq;
    const R st = T::sq(fmax((R)0, (R)1 - ct * ct));
    const R cphi = T::cpi((R)2 * T::u(w[3]));
    const R mu = (R)L.mu;
    const R smu = T::sq(fmax((R)0, (R)1 - mu * mu));
    L.mu = (double)fmin((R)1, fmax((R)-1, mu * ct + smu * st * cphi));
  } else if (ch.kind == EXCITATION) {
    L.eq -= ch.loss_q;
    o.excit += (unsigned long long)ch.loss_q;
  } else if (ch.kind == IONIZATION) {
    const long long avail = L.eq - ch.loss_q;
    const R eps = (R)P.eps_ion;
    const R wmax = (e - (R)ch.loss_ev) * (R)0.5;
    const R wsec = eps * T::tn(T::u(w[2]) * T::atn(wmax * (R)P.inv_eps_ion));
    long long wq = quant_e((double)wsec);
    if (wq > avail / 2) wq = avail / 2;
    if (wq < 0) wq = 0;
    const long long eq1 = avail - wq;
    sadd(&S.ledger[L_LOSS_IONIZ], ch.loss_q);
    // binary encounter: cos^2 of the polar angles are the energy fractions
    const double inv_avail = avail > 0 ? 1.0 / (double)avail : 0.0;
    const R c2p = avail > 0 ? (R)((double)eq1 * inv_avail) : (R)1;
    const R c2s = (R)((double)wq * inv_avail);
    const R cp = T::sq(c2p), sp = T::sq(c2s);
    const R cphi = T::cpi((R)2 * T::u(w[3]));
    const R mu = (R)L.mu;
    const R smu = T::sq(fmax((R)0, (R)1 - mu * mu));
    const R mu_p = fmin((R)1, fmax((R)-1, mu * cp + smu * sp * cphi));
    const R mu_s = fmin((R)1, fmax((R)-1, mu * sp - smu * cp * cphi));
    const unsigned evc = L.ev - 1;
    // slow electron (azimuth opposite to the fast one)
    sadd(&S.ledger[L_BIRTHS + SP_E], 1);
    sadd(&S.ledger[L_N_SPAWN_E], 1);
    Lane c;
    c.z = L.z; c.eq = wq; c.mu = (double)mu_s; c.node = child_node(L.node, evc, 0);
    c.tal = 0.0; c.pid = L.pid; c.ev = 0; c.sp = SP_E; c.j = L.j;
    if (wq < P.ecut_q) die<F32>(P, S, c, R_CUTOFF, L_E_CUTOFF);
    else emit(port, c);
    // ion with a thermal target's velocity (no recoil)
    if (ch.sout >= 0) {
      Lane ion;
      ion.z = L.z; ion.node = child_node(L.node, evc, 1); ion.tal = 0.0; ion.pid = L.pid;
      ion.ev = 0; ion.sp = ch.sout; ion.j = L.j;
      unsigned long long wi[4];
      philox4x64_10(0ULL, ion.node, ((unsigned long long)P.pass << 8) | DOM_ION_BIRTH, 0ULL,
                    P.seed, L.pid, wi);
      thermal<F32>(P, wi, ion.eq, ion.mu);
      sadd(&S.ledger[L_E_IN_THERMAL], ion.eq);
      sadd(&S.ledger[L_BIRTHS + ch.sout], 1);
      sadd(&S.ledger[L_N_SPAWN_ION], 1);
      emit(port, ion);
    }
    L.eq = eq1;
    L.mu = (double)mu_p;
  } else if (ch.kind == CLUSTERING) {
    die<F32>(P, S, L, R_CLUSTER, L_E_CLUSTER);
    unsigned long long wc[4];
    const unsigned evc = L.ev - 1;
    philox4x64_10((unsigned long long)evc, L.node,
                  ((unsigned long long)P.pass << 8) | DOM_CLUSTER, 0ULL, P.seed, L.pid, wc);
    long long eqc;
    double muc;
    thermal<F32>(P, wc, eqc, muc);
    L.node = child_node(L.node, evc, 2);
    L.eq = eqc;
    L.mu = muc;
    L.tal = 0.0;
    L.ev = 0;
    L.sp = ch.sout;
    sadd(&S.ledger[L_E_IN_THERMAL], eqc);
    sadd(&S.ledger[L_BIRTHS + ch.sout], 1);
    return;
  } else {  // RECOMBINATION
    atomicAdd(P.recomb + (size_t)ch.sout * P.nz + jc, 1ULL);
    die<F32>(P, S, L, R_RECOMB, L_E_RECOMB);
    o.alive = false;
    return;
  }
  // ---- terminator (Sec. 3.2) ----
  if (L.sp == SP_E && L.eq < P.ecut_q) {
    die<F32>(P, S, L, R_CUTOFF, L_E_CUTOFF);
    o.alive = false;
  } else if (L.ev >= P.max_coll) {
    die<F32>(P, S, L, R_CAP_COLL, L_E_CAP);
    o.alive = false;
  } else if (P.track_time && L.tal >= P.max_life) {
    die<F32>(P, S, L, R_CAP_TIME, L_E_CAP);
    o.alive = false;
  }
}

// ---------------------------------------------------------------------------
// persistent kernel

// Copy the column tables (and the pass-2 recombination fields) into dynamic
// shared memory when they fit; the event code reads them through P's pointers.
__device__ void stage_tables(Params& SP, const Params& Pk, double* dyn, int dyn_doubles) {
  const int nz = Pk.nz;
  int need = (3 * nz + 2) + (Pk.nq + 1 + 1) / 2 + 1;
  for (int k = 0; k < Pk.nch; ++k)
    if (Pk.fcol[k]) need += 2 * nz + 1;
  if (need > dyn_doubles) return;                   // stay in global memory
  double* col = dyn;
  double* fac = col + (nz + 1);
  double* nseg = fac + (nz + 1);
  int* ginv = (int*)(nseg + nz);
  double* next = (double*)(ginv + ((Pk.nq + 2) & ~1));
  for (int i = threadIdx.x; i <= nz; i += blockDim.x) col[i] = Pk.colgas[i];
  for (int i = threadIdx.x; i <= nz; i += blockDim.x) fac[i] = Pk.faces[i];
  for (int i = threadIdx.x; i < nz; i += blockDim.x) nseg[i] = Pk.nseg[i];
  if (Pk.ginv)
    for (int i = threadIdx.x; i <= Pk.nq; i += blockDim.x) ginv[i] = Pk.ginv[i];
  if (threadIdx.x == 0) {
    SP.colgas = col;
    SP.faces = fac;
    SP.nseg = nseg;
    if (Pk.ginv) SP.ginv = ginv;
  }
  for (int k = 0; k < Pk.nch; ++k) {
    if (!Pk.fcol[k]) continue;
    double* fc = next;
    double* fr = next + (nz + 1);
    next += 2 * nz + 1;
    for (int i = threadIdx.x; i <= nz; i += blockDim.x) fc[i] = Pk.fcol[k][i];
    for (int i = threadIdx.x; i < nz; i += blockDim.x) fr[i] = Pk.frate[k][i];
    if (threadIdx.x == 0) { SP.fcol[k] = fc; SP.frate[k] = fr; }
  }
}

template <bool F32>
__global__ void __launch_bounds__(256) transport_kernel(const Params Pk, Ring R, Control* ctl,
                                                        const volatile int* cancel,
                                                        unsigned long long timeout_ns,
                                                        int dyn_doubles) {
  const unsigned long long deadline = globaltimer_ns() + timeout_ns;
  extern __shared__ double dyn[];
  __shared__ Shared S;
  __shared__ Params SP;
  __shared__ WarpQueue wq[WARPS];
  if (threadIdx.x == 0) SP = Pk;
  for (int i = threadIdx.x; i < LEDGER; i += blockDim.x) S.ledger[i] = 0;
  for (int i = threadIdx.x; i < MAXCH; i += blockDim.x) S.chan[i] = 0;
  if (threadIdx.x < WARPS) wq[threadIdx.x].top = 0;
  __syncthreads();
  stage_tables(SP, Pk, dyn, dyn_doubles);
  __syncthreads();
  const Params& P = SP;

  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  WarpQueue& Q = wq[threadIdx.x >> 5];
  bool has = false;
  Lane L;
  EventOut o;
  o.flights = 0;
  o.colls = 0;
  o.recoil = 0;
  o.excit = 0;
  o.chan = -1;
  unsigned long long started = 0;
  unsigned long long idle_iters = 0, busy_iters = 0, busy_lane_iters = 0;
  unsigned idle_ns = 128;
  RingPort port;
  port.R = &R;
  port.ctl = ctl;
  port.deadline = deadline;
  port.q = &Q;
  port.local = true;
  port.spilled = 0;

  for (long long iter = 0;; ++iter) {
    if ((iter & 63) == 0) {
      int stop = 0;
      if (lane == 0) {
        if (ld_relaxed_i(&ctl->abort)) stop = 1;
        else if (cancel && ld_relaxed_i((const int*)cancel)) {
          atomicCAS(&ctl->error, 0, ERR_CANCELLED);
          atomicExch(&ctl->abort, 1);
          stop = 1;
        } else if (globaltimer_ns() > deadline) {
          atomicCAS(&ctl->error, 0, ERR_TIMEOUT);
          atomicExch(&ctl->abort, 1);
          stop = 1;
        }
      }
      if (__shfl_sync(FULL, stop, 0)) break;
      port.local = ld_relaxed(&ctl->prim_next) < (unsigned long long)P.n_prim;
    }

    // ---- idle lanes take the warp's own products first (newest first) ----
    __syncwarp();
    {
      const unsigned need0 = __ballot_sync(FULL, !has);
      int top = Q.top;
      if (top > WQ) top = WQ;
      const int take = min(__popc(need0), top);
      if (!has) {
        const int rank = __popc(need0 & lt);
        if (rank < take) {
          L = Q.s[top - 1 - rank];
          has = true;
          started += 1;
        }
      }
      int left = top - take;
      // once the primaries are used up, move what is left to the shared ring
      // where idle warps can take it (counted there instead of here)
      if (!port.local && left > 0) {
        unsigned long long pos = 0;
        if (lane == 0) pos = atomicAdd(&ctl->tail, (unsigned long long)left);
        pos = __shfl_sync(FULL, pos, 0);
        if (lane < left) ring_put(R, ctl, pos + lane, Q.s[lane], deadline);
        __syncwarp();
        if (lane == 0) {
          __threadfence();
          atomicAdd((unsigned long long*)&ctl->active, (unsigned long long)(-(long long)left));
          port.spilled += left;
        }
        left = 0;
      }
      __syncwarp();
      if (lane == 0) Q.top = left;
      __syncwarp();
    }

    // ---- other idle lanes take work: products from the ring, then primaries ----
    const unsigned need = __ballot_sync(FULL, !has);
    if (need) {
      const int k = __popc(need);
      unsigned long long base = 0;
      int got = 0, src = 0;
      if (lane == 0) {
        // Count the lanes as active only when work is visible, then claim it:
        // idle warps that find nothing leave the counter alone.
        unsigned long long h = ld_relaxed(&ctl->head), t = ld_relaxed(&ctl->tail);
        const unsigned long long pn = ld_relaxed(&ctl->prim_next);
        const bool ring_work = h < t;
        const bool prim_work = pn < (unsigned long long)P.n_prim && t - h < R.cap / 4;
        if (ring_work || prim_work) {
          atomicAdd((unsigned long long*)&ctl->active, (unsigned long long)k);
          __threadfence();
          for (int tries = 0; tries < 16 && h < t; ++tries) {
            unsigned long long take = t - h < (unsigned long long)k ? t - h : (unsigned long long)k;
            unsigned long long old = atomicCAS(&ctl->head, h, h + take);
            if (old == h) { base = h; got = (int)take; src = 1; break; }
            h = old;
            t = ld_relaxed(&ctl->tail);
          }
          if (got == 0 && prim_work) {
            unsigned long long p0 = atomicAdd(&ctl->prim_next, (unsigned long long)k);
            if (p0 < (unsigned long long)P.n_prim) {
              unsigned long long left = (unsigned long long)P.n_prim - p0;
              base = p0;
              got = left < (unsigned long long)k ? (int)left : k;
              src = 2;
            }
          }
          if (got < k) atomicAdd((unsigned long long*)&ctl->active, (unsigned long long)(got - k));
        }
      }
      base = __shfl_sync(FULL, base, 0);
      got = __shfl_sync(FULL, got, 0);
      src = __shfl_sync(FULL, src, 0);
      bool born_dead = false;
      if (!has && got > 0) {
        const int rank = __popc(need & lt);
        if (rank < got) {
          const unsigned long long idx = base + rank;
          if (src == 1) {
            has = ring_get(R, ctl, idx, L, deadline);
          } else {
            L.z = P.pz[idx];
            L.eq = quant_e(P.pe[idx]);
            L.mu = P.pmu[idx];
            L.sp = P.psp[idx];
            L.node = 0;
            L.tal = 0.0;
            L.ev = 0;
            L.pid = (unsigned long long)P.pid_offset + idx;
            L.j = segment_of(P, L.z);
            sadd(&S.ledger[L_E_IN_PRIMARY], L.eq);
            sadd(&S.ledger[L_BIRTHS + L.sp], 1);
            if (L.sp == SP_E && L.eq < P.ecut_q) {
              die<F32>(P, S, L, R_CUTOFF, L_E_CUTOFF);
              born_dead = true;
            } else {
              has = true;
            }
          }
          started += 1;
        }
      }
      const unsigned md = __ballot_sync(FULL, born_dead);
      if (md && lane == 0) {
        __threadfence();
        atomicAdd((unsigned long long*)&ctl->active, (unsigned long long)(-(long long)__popc(md)));
      }
    }

    const unsigned busy = __ballot_sync(FULL, has);
    if (!busy) {
      int done = 0;
      if (lane == 0) {
        // Done when no work is queued, none will come (no particle is held),
        // and nothing moved between two snapshots taken around the read of
        // the active count.  A claim visible in the first snapshot makes its
        // active increment visible; a product reserved by a particle whose
        // death is visible shows up in the second snapshot.
        const unsigned long long h1 = ld_relaxed(&ctl->head), t1 = ld_relaxed(&ctl->tail);
        const unsigned long long p1 = ld_relaxed(&ctl->prim_next);
        __threadfence();
        const long long a = ld_relaxed_s(&ctl->active);
        __threadfence();
        const unsigned long long h2 = ld_relaxed(&ctl->head), t2 = ld_relaxed(&ctl->tail);
        const unsigned long long p2 = ld_relaxed(&ctl->prim_next);
        done = (a <= 0 && h1 == h2 && t1 == t2 && p1 == p2 && h1 >= t1 &&
                p1 >= (unsigned long long)P.n_prim);
      }
      if (__shfl_sync(FULL, done, 0)) break;
      __nanosleep(idle_ns);
      if (idle_ns < 4096) idle_ns <<= 1;
      ++idle_iters;
      continue;
    }
    idle_ns = 128;
    busy_lane_iters += __popc(busy);
    ++busy_iters;

    // ---- one event ----
    bool died = false;
    if (has) {
      event<F32>(P, S, L, o, port);
      if (!o.alive) { has = false; died = true; }
    }
    __syncwarp();
    if (lane == 0 && Q.top > WQ) Q.top = WQ;          // pushes past the end went to the ring

    // ---- channel counts, one shared-memory add per distinct channel per warp ----
    const unsigned mc = __ballot_sync(FULL, o.chan >= 0);
    if (o.chan >= 0) {
      const unsigned grp = __match_any_sync(mc, o.chan);
      if (lane == __ffs(grp) - 1) atomicAdd(&S.chan[o.chan], (unsigned long long)__popc(grp));
    }
    o.chan = -1;

    const unsigned md = __ballot_sync(FULL, died);
    if (md) {
      __threadfence();
      if (lane == 0)
        atomicAdd((unsigned long long*)&ctl->active, (unsigned long long)(-(long long)__popc(md)));
    }
  }

  // ---- flush per-lane and per-block counters ----
  unsigned long long f = o.flights, c = o.colls, st = started, rc = o.recoil, ex = o.excit;
  unsigned long long sp = port.spilled;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    sp += __shfl_down_sync(FULL, sp, off);
    f += __shfl_down_sync(FULL, f, off);
    c += __shfl_down_sync(FULL, c, off);
    st += __shfl_down_sync(FULL, st, off);
    rc += __shfl_down_sync(FULL, rc, off);
    ex += __shfl_down_sync(FULL, ex, off);
  }
  if (lane == 0) {
    atomicAdd(&ctl->idle_iters, idle_iters);
    atomicAdd(&ctl->spilled, sp);
    atomicAdd(&ctl->busy_iters, busy_iters);
    atomicAdd(&ctl->busy_lane_iters, busy_lane_iters);
    atomicAdd(&S.ledger[L_N_FLIGHT], f);
    atomicAdd(&S.ledger[L_N_COLL], c);
    atomicAdd(&S.ledger[L_LOSS_RECOIL], rc);
    atomicAdd(&S.ledger[L_LOSS_EXCIT], ex);
    atomicAdd(&ctl->particles, st);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < LEDGER; i += blockDim.x)
    if (S.ledger[i]) atomicAdd(P.ledger + i, S.ledger[i]);
  for (int i = threadIdx.x; i < P.nch; i += blockDim.x)
    if (S.chan[i]) atomicAdd(P.chan_count + i, S.chan[i]);
}

// ---------------------------------------------------------------------------
// host-callable launchers (used by the C ABI in karl_abi.cu)

// dynamic shared memory for the staged tables: at most this much per block
constexpr int DYN_MAX_BYTES = 120 * 1024;

// Doubles of dynamic shared memory the staged tables of P need (0: too big,
// read them from global memory).
int transport_dyn_doubles(const Params& P) {
  int need = (3 * P.nz + 2) + (P.nq + 1 + 1) / 2 + 1;
  for (int k = 0; k < P.nch; ++k)
    if (P.fcol[k]) need += 2 * P.nz + 1;
  return need * 8 <= DYN_MAX_BYTES ? need : 0;
}

cudaError_t launch_transport(bool f32, const Params& P, const Ring& R, Control* ctl,
                             const volatile int* cancel, unsigned long long timeout_ns, int grid,
                             int block, cudaStream_t st) {
  const int dd = transport_dyn_doubles(P);
  const size_t bytes = (size_t)dd * 8;
  if (f32)
    transport_kernel<true><<<grid, block, bytes, st>>>(P, R, ctl, cancel, timeout_ns, dd);
  else
    transport_kernel<false><<<grid, block, bytes, st>>>(P, R, ctl, cancel, timeout_ns, dd);
  return cudaGetLastError();
}

cudaError_t transport_setup() {
  cudaError_t e = cudaFuncSetAttribute(transport_kernel<true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, DYN_MAX_BYTES);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(transport_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              DYN_MAX_BYTES);
}

cudaError_t transport_occupancy(bool f32, const Params& P, int block, int* blocks_per_sm) {
  const size_t bytes = (size_t)transport_dyn_doubles(P) * 8;
  if (f32)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, transport_kernel<true>,
                                                         block, bytes);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, transport_kernel<false>,
                                                       block, bytes);
}

}  // namespace karl
