// event.cuh - one transport event of one particle, shared by the single-run
// and the multi-request (batched / served) kernels.
//
// A free flight by optical depth (Eqs. mean_free_path and distance_from_mfp
// over the piecewise-constant column, equal in law to the segment-stop mover
// of Sec. 3.1), the time/density and current tallies of Secs. 2.2-2.3 as
// range adds, the terminator of Sec. 3.2, a channel chosen with probability
// sigma_i n_i / sum_j sigma_j n_j, and its kinematics (Sec. 3.3).
#pragma once
#include <cooperative_groups.h>

#include "karl_device.cuh"

namespace karl {


constexpr double Q_E = 16777216.0;             // 2^24 energy units per eV
constexpr double INV_Q_E = 1.0 / 16777216.0;
constexpr double Q_T = 1125899906842624.0;     // 2^50 time units per s
constexpr double C_LIGHT = 299792458.0;
constexpr unsigned FULL = 0xffffffffu;
constexpr long long SPIN_LIMIT = 1LL << 26;    // bounded waits on ring cells

// Explicitly rounded products and fused multiply-adds.  Every product that
// feeds a sum in the event is written with these, so the compiler cannot fuse
// a multiply into an add in one kernel and not in another: the single-run and
// the multi-request kernels then give the same bits.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// float <-> double of the FP32 form (the conversions: building them from the
// bits measured slower there); identities for FP64
__device__ __forceinline__ double to_d(double x) { return x; }
__device__ __forceinline__ double to_d(float x) { return (double)x; }
template <class R> __device__ __forceinline__ R from_d(double x);
template <> __device__ __forceinline__ double from_d<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_d<float>(double x) { return (float)x; }

template <bool F32> struct RT;
template <> struct RT<false> {
  using R = double;
  static __device__ __forceinline__ R u(unsigned long long w) { return u01d(w); }
  static __device__ __forceinline__ R eta(unsigned long long w) { return eta01d(w); }
  static __device__ __forceinline__ R lg(R x) { return log_tab(x); }
  static __device__ __forceinline__ R sq(R x) { return sqrt(x); }
  static __device__ __forceinline__ R rsq(R x) { return rsqrt(x); }
  static __device__ __forceinline__ R tn(R x) { return tan(x); }
  static __device__ __forceinline__ R atn(R x) { return atan(x); }
  static __device__ __forceinline__ R cpi(R x) { return cospi(x); }
  static __device__ __forceinline__ R max0(R x) { return dmax0(x); }
  static __device__ __forceinline__ R clamp1(R x) { return dclamp1(x); }
  static __device__ __forceinline__ R spi(R x) { return sinpi(x); }
  // value and slope to the next node of channel k at node i ([node][channel][2])
  static __device__ __forceinline__ void tab2(const Params& P, int k, int i, R& a, R& s) {
    const double2 t = __ldg((const double2*)P.sig + (size_t)i * P.nch + k);
    a = t.x;
    s = t.y;
  }
  // cumulative value and slope of the species' gas channels 0..c at node i
  static __device__ __forceinline__ void cum2(const Params& P, int s, int i, int c, R& a, R& sl) {
    const double2 t = __ldg((const double2*)P.cum + P.cum_off[s] + (size_t)i * P.ncg[s] + c);
    a = t.x;
    sl = t.y;
  }
  static __device__ __forceinline__ R angp(const Params& P, size_t i) { return __ldg(P.ang_pdf + i); }
  static __device__ __forceinline__ R angc(const Params& P, size_t i) { return __ldg(P.ang_cum + i); }
  // eq 2^-24, built from the bits of eq (exact; no FP64 conversion or multiply)
  static __device__ __forceinline__ R energy(long long eq) {
    return eq >= 0 && eq < (1LL << 53) ? u53_scaled((unsigned long long)eq, 24)
                                       : (double)eq * (1.0 / 16777216.0);
  }
  static __device__ __forceinline__ long long quant_de(R de) {   // de >= 0
    return trunc_nonneg(de * 16777216.0 + 0.5);
  }
  // a transfer of either sign, rounded to the nearest 2^-24 eV
  static __device__ __forceinline__ long long quant_signed(R de) {
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
  static __device__ __forceinline__ R max0(R x) { return fmaxf(0.0f, x); }
  static __device__ __forceinline__ R clamp1(R x) { return fminf(1.0f, fmaxf(-1.0f, x)); }
  static __device__ __forceinline__ R spi(R x) { return sinpif(x); }
  static __device__ __forceinline__ void tab2(const Params& P, int k, int i, R& a, R& s) {
    const float2 t = __ldg((const float2*)P.sigf + (size_t)i * P.nch + k);
    a = t.x;
    s = t.y;
  }
  static __device__ __forceinline__ void cum2(const Params& P, int s, int i, int c, R& a, R& sl) {
    const float2 t = __ldg((const float2*)P.cumf + P.cum_off[s] + (size_t)i * P.ncg[s] + c);
    a = t.x;
    sl = t.y;
  }
  static __device__ __forceinline__ R angp(const Params& P, size_t i) { return __ldg(P.ang_pdff + i); }
  static __device__ __forceinline__ R angc(const Params& P, size_t i) { return __ldg(P.ang_cumf + i); }
  // energy from 2^-24 eV units with 32-bit conversions (below 65 keV; exact
  // to FP32 rounding below 256 eV, where thermal energies live)
  static __device__ __forceinline__ R energy(long long eq) {
    if (eq < (1LL << 32)) return (float)(unsigned)eq * (1.0f / 16777216.0f);
    return eq < (1LL << 40) ? (float)(unsigned)(eq >> 8) * (1.0f / 65536.0f)
                            : (float)eq * (1.0f / 16777216.0f);
  }
  static __device__ __forceinline__ long long quant_signed(R de) {
    return (long long)floorf(de * 16777216.0f + 0.5f);
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
  int slot;                     // request slot (multi-request kernel; 0 otherwise)
};

// segment (20 bits) | species (2 bits) | request slot (10 bits) in one ring word
__device__ __forceinline__ unsigned pack_sj(const Lane& p) {
  return (unsigned)p.j | ((unsigned)p.sp << 20) | ((unsigned)p.slot << 22);
}
__device__ __forceinline__ void unpack_sj(unsigned w, Lane& p) {
  p.j = (int)(w & 0xfffffu);
  p.sp = (int)((w >> 20) & 3u);
  p.slot = (int)(w >> 22);
}

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

// 1 / v for kinetic energy e (relativistic: v = c sqrt(x (2 + x)) / (1 + x),
// x = e / m c^2); every use of the speed divides by it
template <bool F32>
__device__ __forceinline__ typename RT<F32>::R inv_speed(typename RT<F32>::R e,
                                                         typename RT<F32>::R inv_m) {
  using R = typename RT<F32>::R;
  const R x = e * inv_m;
  return ((R)1 + x) * RT<F32>::rsq(x * ((R)2 + x)) * (R)(1.0 / C_LIGHT);
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

static __device__ bool ring_put(const Ring& R, Control* ctl, unsigned long long pos, const Lane& p,
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
  R.pid[i] = p.pid; R.ev[i] = p.ev; R.sj[i] = pack_sj(p);
  st_release(cell, pos + 1);
  return true;
}

static __device__ bool ring_get(const Ring& R, Control* ctl, unsigned long long pos, Lane& p,
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
  unpack_sj(R.sj[i], p);
  st_release(cell, pos + R.cap);
  return true;
}

// ---------------------------------------------------------------------------
// one event of one particle

struct EventOut {
  bool alive;
  bool parked;                            // handed to the warp's batch of rare collisions
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
constexpr int WARPS = 8;                  // multi-request kernel: blocks of up to 256 threads
struct WarpQueue {
  Lane s[WQ];
  int top;
};

// Collisions in the rare channels (ionization with its products, clustering,
// charge exchange) cost as much FP64 work as a whole ordinary event, and a warp pays that cost
// in full for a single lane.  A lane that selects one parks its particle here
// (state after the flight, channel chosen) and takes other work; when enough
// have gathered the whole warp performs them together.  The kinematics draw
// from the same counter-based stream either way, so results do not change.
// The same slots also hold, from the top down, the particles busy lanes hand
// back to make room for a batch; free lanes resume those before other work.
constexpr int RB = 32;                    // parked collisions per warp
constexpr int RB_TRIGGER = 24;            // batch size that starts a batch
struct RareBuf {
  Lane s[RB];
  int8_t ch[RB];
  int n;                                  // parked: slots [0, n)
  int r;                                  // handed back: slots [RB - r, RB)
};

struct RingPort {
  const Ring* R;
  Control* ctl;
  unsigned long long deadline;
  WarpQueue* q;
  RareBuf* rare;           // NULL: perform rare collisions in line
  bool local;              // primaries remain: keep products in the warp queue
  unsigned long long spilled;
  // multi-request kernel: every existing particle counts in its slot's live
  // word (low 32 bits); NULL in the single-run kernel
  unsigned long long* slot_live;
};

// Lanes that emit a product together take their queue slots, and past the
// queue's end their ring cells, with one atomic per warp: the first lane of
// the group reserves a range and every lane writes at its rank in the group.
__device__ __forceinline__ void emit(RingPort& port, const Lane& p) {
  namespace cg = cooperative_groups;
  if (port.slot_live) atomicAdd(port.slot_live, 1ULL);
  bool placed = false;
  if (port.local) {                        // uniform over the warp
    cg::coalesced_group g = cg::coalesced_threads();
    const int n = (int)g.size();
    int base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(&port.q->top, n);
    base = g.shfl(base, 0);
    const int i = base + (int)g.thread_rank();
    if (i < WQ) {
      port.q->s[i] = p;
      placed = true;
    }
    const int kept = base >= WQ ? 0 : min(WQ - base, n);
    if (!port.slot_live && g.thread_rank() == 0 && kept > 0)
      atomicAdd((unsigned long long*)&port.ctl->active, (unsigned long long)kept);  // held by this warp
  }
  if (!placed) {
    cg::coalesced_group g = cg::coalesced_threads();
    unsigned long long base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(&port.ctl->tail, (unsigned long long)g.size());
    base = g.shfl(base, 0);
    ring_put(*port.R, port.ctl, base + g.thread_rank(), p, port.deadline);
    port.spilled += 1;
  }
}

template <bool F32>
__device__ __forceinline__ void die(const Params& P, unsigned long long* led, Lane& L, int reason,
                                    int slot) {
  sadd(led + L_DEATHS + L.sp * NREASON + reason, 1);
  sadd(led + slot, L.eq);
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

// cos(chi) of an elastic collision from the angle table `set` at impact
// energy e (Sec. 3.3 Elastic: the energy bin of the table is chosen and the
// angle drawn from its piecewise-linear distribution).  The bin is the
// log-spaced one holding e, clamped to the first and last.  With the pdf p_i
// at x_i = -1 + i h and its cumulative integral C_i, t = u C_(n-1) falls in
// the interval [x_i, x_i+1] of the largest i with C_i <= t (binary search),
// and cos chi = x_i + s with s in [0, h] the root of
// C_i + p_i s + (p_i+1 - p_i) s^2 / (2h) = t, taken in the form
// s = 2r / (p_i + sqrt(p_i^2 + 2 r (p_i+1 - p_i) / h)), r = t - C_i, which
// stays accurate when the pdf is flat.
template <bool F32>
__device__ __noinline__ typename RT<F32>::R table_cchi(const Params& P, int set,
                                                       typename RT<F32>::R e,
                                                       typename RT<F32>::R u) {
  using T = RT<F32>;
  using R = typename T::R;
  const int nb = P.ang_nb, n = P.ang_nmu;
  int b = (int)floor(T::lg(e * (R)P.ang_inv_lo[set]) * (R)P.ang_scale[set]);
  b = b < 0 ? 0 : (b > nb - 1 ? nb - 1 : b);
  const size_t row = ((size_t)set * nb + b) * n;
  const R t = u * T::angc(P, row + n - 1);
  int lo = 0, hi = n - 1;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (T::angc(P, row + mid) <= t) lo = mid; else hi = mid;
  }
  const R h = (R)P.ang_h;
  const R r = t - T::angc(P, row + lo);
  const R a = T::angp(P, row + lo);
  const R slope = (T::angp(P, row + lo + 1) - a) * (R)P.ang_inv_h;
  const R den = a + T::sq(fmax((R)0, a * a + (R)2 * slope * r));
  R sv = den > (R)0 ? (R)2 * r / den : (R)0;
  sv = fmin(fmax(sv, (R)0), h);
  return fmin((R)1, (R)-1 + (R)lo * h + sv);
}

// cos(chi) of an elastic collision of channel ch at impact energy e for the
// uniform u: isotropic (2u - 1) without a table or below its threshold.
template <bool F32>
__device__ __forceinline__ typename RT<F32>::R elastic_cchi(const Params& P, const ChanDev& ch,
                                                            typename RT<F32>::R e,
                                                            typename RT<F32>::R u) {
  using R = typename RT<F32>::R;
  if (ch.ang >= 0 && e >= (R)P.ang_thr[ch.ang]) return table_cchi<F32>(P, ch.ang, e, u);
  return (R)2 * u - (R)1;
}

// Elastic collision with a moving target (Sec. 3.3 Elastic: the target moves
// with the gas drift plus a Maxwell-Boltzmann velocity; the impactor turns in
// the centre-of-mass frame).  Nonrelativistic velocities in units of c; the
// impactor's gyrophase is taken as 0 (the target distribution is symmetric
// about z).  Targets are met at a rate proportional to the relative speed, so
// the thermal part w of the target velocity (gas frame, impactor velocity u)
// is drawn from |u - w| f(w) by the free-gas rejection method: speed from the
// mixture (|u| + s) s^2 exp(-s^2/2a^2) -- a Maxwell speed with probability
// |u| sqrt(pi) / (|u| sqrt(pi) + 2 sqrt(2) a), else s^2/2a^2 ~ Gamma(2) --,
// isotropic direction, accepted with probability |u - w| / (|u| + s); attempt
// k draws blocks 2k and 2k+1 of the collision's DOM_TARGET stream, and after
// 64 rejections the last draw stands.  The centre-of-mass polar angle (cos
// uniform, w[2]) and azimuth (w[3], from the plane of z and the relative
// velocity) turn the relative velocity.
// The thermal part (wx, wy, wz) of the target velocity met by an impactor of
// velocity (v1x, 0, v1z) (units of c), drawn as described above.
template <bool F32>
__device__ __forceinline__ void draw_target(const Params& P, const Lane& L,
                                            typename RT<F32>::R v1x, typename RT<F32>::R v1z,
                                            typename RT<F32>::R& wx, typename RT<F32>::R& wy,
                                            typename RT<F32>::R& wz,
                                            unsigned long long sub0 = 0) {
  using T = RT<F32>;
  using R = typename T::R;
  const R a = (R)P.target_a, ud = (R)P.drift_c;
  const R uz = v1z - ud;
  const R un = T::sq(v1x * v1x + uz * uz);
  const R rpi = (R)1.7724538509055160273, r8 = (R)2.8284271247461900976;
  const R pmax = un * rpi / (un * rpi + r8 * a);
  wx = (R)0; wy = (R)0; wz = (R)0;
  for (int k = 0; k < 64; ++k) {
    unsigned long long b0[4], b1[4];
    const unsigned long long ctr2 = ((unsigned long long)P.pass << 8) | DOM_TARGET;
    philox4x64_10((unsigned long long)(L.ev - 1), L.node, ctr2, sub0 + 2ULL * k, P.seed, L.pid,
                  b0);
    philox4x64_10((unsigned long long)(L.ev - 1), L.node, ctr2, sub0 + 2ULL * k + 1, P.seed,
                  L.pid, b1);
    const R l1 = -T::lg(T::eta(b0[1])), l2 = -T::lg(T::eta(b0[2]));
    R s2;
    if (T::u(b0[0]) < pmax) {
      const R c = T::cpi((R)2 * T::u(b0[3]));
      s2 = a * a * ((R)2 * l1 + (R)2 * l2 * c * c);     // chi-square, 3 degrees of freedom
    } else {
      s2 = (R)2 * a * a * (l1 + l2);                     // Gamma(2, 1)
    }
    const R sp = T::sq(s2);
    const R ct = (R)2 * T::u(b1[0]) - (R)1;
    const R st = T::sq(fmax((R)0, (R)1 - ct * ct));
    const R ph = (R)2 * T::u(b1[1]);
    wx = sp * st * T::cpi(ph);
    wy = sp * st * T::spi(ph);
    wz = sp * ct;
    const R g0 = v1x - wx, g1 = -wy, g2 = uz - wz;
    const R gn = T::sq(g0 * g0 + g1 * g1 + g2 * g2);
    if (T::u(b1[2]) * (un + sp) < gn) break;
  }
}

template <bool F32>
__device__ __noinline__ void moving_target_elastic(const Params& P, const ChanDev& ch, Lane& L,
                                                   const unsigned long long w[4],
                                                   unsigned long long& recoil) {
  using T = RT<F32>;
  using R = typename T::R;
  const int s = L.sp;
  const R m1 = (R)P.mass[s], m2 = (R)P.target_mass, M = m1 + m2;
  const R e = T::energy(L.eq);
  const R s1 = T::sq((R)2 * e / m1);
  const R mu = (R)L.mu;
  const R sperp = T::sq(fmax((R)0, (R)1 - mu * mu));
  const R v1x = s1 * sperp, v1z = s1 * mu;
  R wx, wy, wz;
  draw_target<F32>(P, L, v1x, v1z, wx, wy, wz);
  const R v2x = wx, v2y = wy, v2z = (R)P.drift_c + wz;
  // centre-of-mass velocity and relative velocity
  const R Vx = (m1 * v1x + m2 * v2x) / M, Vy = (m2 * v2y) / M, Vz = (m1 * v1z + m2 * v2z) / M;
  const R gx = v1x - v2x, gy = -v2y, gz = v1z - v2z;
  const R gn = T::sq(gx * gx + gy * gy + gz * gz);
  R hx = (R)0, hy = (R)0, hz = (R)1;
  if (gn > (R)0) { hx = gx / gn; hy = gy / gn; hz = gz / gn; }
  // e1: the part of z perpendicular to g (x if g is along z); e2 = h x e1
  R ax = -hz * hx, ay = -hz * hy, az = (R)1 - hz * hz;
  R n1 = T::sq(ax * ax + ay * ay + az * az);
  if (n1 < (R)1e-12) { ax = (R)1; ay = (R)0; az = (R)0; n1 = (R)1; }
  ax /= n1; ay /= n1; az /= n1;
  const R bx = hy * az - hz * ay, by = hz * ax - hx * az, bz = hx * ay - hy * ax;
  // impact energy: the impactor's kinetic energy relative to the target
  const R cchi = elastic_cchi<F32>(P, ch, (R)0.5 * m1 * gn * gn, T::u(w[2]));
  const R schi = T::sq(fmax((R)0, (R)1 - cchi * cchi));
  const R phi = (R)2 * T::u(w[3]);
  const R cph = T::cpi(phi), sph = T::spi(phi);
  const R f = m2 / M * gn;
  const R nx = Vx + f * (schi * cph * ax + schi * sph * bx + cchi * hx);
  const R ny = Vy + f * (schi * cph * ay + schi * sph * by + cchi * hy);
  const R nz = Vz + f * (schi * cph * az + schi * sph * bz + cchi * hz);
  const R sp2 = nx * nx + ny * ny + nz * nz;
  const R e1 = (R)0.5 * m1 * sp2;
  long long rq = T::quant_signed(e - e1);          // energy given to the gas (either sign)
  if (rq > L.eq) rq = L.eq;
  recoil += (unsigned long long)rq;
  L.eq -= rq;
  L.mu = sp2 > (R)0 ? (double)fmin((R)1, fmax((R)-1, nz * T::rsq(sp2))) : 1.0;
}

// Charge exchange (Sec. 3.3 Charge exchange): the ion takes the velocity v2 of
// a target particle drawn as for a moving elastic target (draw_target plus
// the gas drift); its kinetic energy becomes 1/2 m1 |v2|^2 (nonrelativistic)
// and the difference, of either sign, goes to the gas; species unchanged.
template <bool F32>
__device__ __noinline__ void charge_exchange(const Params& P, Lane& L, unsigned long long& recoil) {
  using T = RT<F32>;
  using R = typename T::R;
  const R m1 = (R)P.mass[L.sp];
  const R e = T::energy(L.eq);
  const R s1 = T::sq((R)2 * e / m1);
  const R mu = (R)L.mu;
  const R sperp = T::sq(fmax((R)0, (R)1 - mu * mu));
  R wx, wy, wz;
  draw_target<F32>(P, L, s1 * sperp, s1 * mu, wx, wy, wz);
  const R vz = (R)P.drift_c + wz;
  const R sp2 = wx * wx + wy * wy + vz * vz;
  const R e1 = (R)0.5 * m1 * sp2;
  long long rq = T::quant_signed(e - e1);
  if (rq > L.eq) rq = L.eq;
  recoil += (unsigned long long)rq;
  L.eq -= rq;
  L.mu = sp2 > (R)0 ? (double)fmin((R)1, fmax((R)-1, vz * T::rsq(sp2))) : 1.0;
}

// Terminator of Sec. 3.2 after a collision.
template <bool F32>
__device__ __forceinline__ void terminate(const Params& P, unsigned long long* led, Lane& L,
                                          EventOut& o) {
  if (L.sp == SP_E && L.eq < P.ecut_q) {
    die<F32>(P, led, L, R_CUTOFF, L_E_CUTOFF);
    o.alive = false;
  } else if (L.ev >= P.max_coll) {
    die<F32>(P, led, L, R_CAP_COLL, L_E_CAP);
    o.alive = false;
  } else if (P.track_time && L.tal >= P.max_life) {
    die<F32>(P, led, L, R_CAP_TIME, L_E_CAP);
    o.alive = false;
  }
}

// Ionization with a moving target (Sec. 3.3 Ionization).  The target velocity
// is drawn as for a moving elastic target (draw_target, blocks from 128 r for
// redraw r) and redrawn while the impact energy -- the impactor's kinetic
// energy relative to the target, m1 |v1 - v2|^2 / 2 -- is not above the
// ionization energy I; after 64 redraws the target is taken at rest (its
// impact energy is the lab energy, above I since the channel was chosen).  In
// the target's frame the impact energy is shared as for a target at rest
// (slow electron W from the truncated 1/(1+(W/eps)^2) law on [0, (E_i-I)/2],
// binary-encounter polar angles about the relative velocity, azimuths phi and
// phi - pi from the plane of z and the relative velocity); adding v2 takes
// both electrons back to the lab, and the ion leaves with v2 (no recoil).
// The lab energy the gas gives or takes goes to the recoil ledger (either
// sign), so the ledger stays exact.  Nonrelativistic velocities in units of c.
template <bool F32>
__device__ __noinline__ void moving_target_ionization(const Params& P, unsigned long long* led,
                                                      Lane& L, EventOut& o, RingPort& port,
                                                      int k, const unsigned long long w[4]) {
  using T = RT<F32>;
  using R = typename T::R;
  const ChanDev ch = P.ch[k];
  const int s = L.sp;
  const R m1 = (R)P.mass[s], me = (R)P.mass[SP_E];
  const R e = T::energy(L.eq);
  const R ion_e = (R)ch.loss_ev;
  const R s1 = T::sq((R)2 * e / m1);
  const R mu = (R)L.mu;
  const R sperp = T::sq(fmax((R)0, fma_rn(-mu, mu, (R)1)));
  const R v1x = mul_rn(s1, sperp), v1z = mul_rn(s1, mu);
  R v2x = (R)0, v2y = (R)0, v2z = (R)0, gx = v1x, gy = (R)0, gz = v1z, ei = e;
  for (int r = 0; r < 64; ++r) {
    R wx, wy, wz;
    draw_target<F32>(P, L, v1x, v1z, wx, wy, wz, 128ULL * (unsigned long long)r);
    const R tz = (R)P.drift_c + wz;
    const R dx = v1x - wx, dy = -wy, dz = v1z - tz;
    const R er = mul_rn((R)0.5 * m1, fma_rn(dx, dx, fma_rn(dy, dy, mul_rn(dz, dz))));
    if (er > ion_e) {
      v2x = wx; v2y = wy; v2z = tz;
      gx = dx; gy = dy; gz = dz;
      ei = er;
      break;
    }
  }
  // energy sharing in the target's frame
  const R avail = ei - ion_e;
  const R eps = (R)P.eps_ion;
  const R wmax = (R)0.5 * avail;
  R wsec = eps * T::tn(T::u(w[2]) * T::atn(wmax * (R)P.inv_eps_ion));
  wsec = fmin(fmax(wsec, (R)0), wmax);
  const R e1 = avail - wsec;
  const R cp = T::sq(e1 / avail), sp = T::sq(wsec / avail);
  // basis: h along the relative velocity, b1 the part of z perpendicular to
  // it (x if it is along z), b2 = h x b1
  const R gn = T::sq(fma_rn(gx, gx, fma_rn(gy, gy, mul_rn(gz, gz))));
  R hx = (R)0, hy = (R)0, hz = (R)1;
  if (gn > (R)0) { hx = gx / gn; hy = gy / gn; hz = gz / gn; }
  R ax = -hz * hx, ay = -hz * hy, az = fma_rn(-hz, hz, (R)1);
  R n1 = T::sq(fma_rn(ax, ax, fma_rn(ay, ay, mul_rn(az, az))));
  if (n1 < (R)1e-12) { ax = (R)1; ay = (R)0; az = (R)0; n1 = (R)1; }
  ax /= n1; ay /= n1; az /= n1;
  const R bx = hy * az - hz * ay, by = hz * ax - hx * az, bz = hx * ay - hy * ax;
  const R phi = (R)2 * T::u(w[3]);
  const R cph = T::cpi(phi), sph = T::spi(phi);
  const R u1 = T::sq((R)2 * e1 / m1), u2 = T::sq((R)2 * wsec / me);
  const R sx = fma_rn(cph, ax, mul_rn(sph, bx)), sy = fma_rn(cph, ay, mul_rn(sph, by)),
          sz = fma_rn(cph, az, mul_rn(sph, bz));
  const R ax1 = v2x + u1 * fma_rn(cp, hx, mul_rn(sp, sx));
  const R ay1 = v2y + u1 * fma_rn(cp, hy, mul_rn(sp, sy));
  const R az1 = v2z + u1 * fma_rn(cp, hz, mul_rn(sp, sz));
  const R ax2 = v2x + u2 * fma_rn(sp, hx, -mul_rn(cp, sx));
  const R ay2 = v2y + u2 * fma_rn(sp, hy, -mul_rn(cp, sy));
  const R az2 = v2z + u2 * fma_rn(sp, hz, -mul_rn(cp, sz));
  const R qa = fma_rn(ax1, ax1, fma_rn(ay1, ay1, mul_rn(az1, az1)));
  const R qb = fma_rn(ax2, ax2, fma_rn(ay2, ay2, mul_rn(az2, az2)));
  const R q2 = fma_rn(v2x, v2x, fma_rn(v2y, v2y, mul_rn(v2z, v2z)));
  const long long eq1 = quant_e((double)((R)0.5 * m1 * qa));
  const long long wq = quant_e((double)((R)0.5 * me * qb));
  const R mu1 = qa > (R)0 ? fmin((R)1, fmax((R)-1, az1 * T::rsq(qa))) : (R)1;
  const R mu2 = qb > (R)0 ? fmin((R)1, fmax((R)-1, az2 * T::rsq(qb))) : (R)1;
  sadd(led + L_LOSS_IONIZ, ch.loss_q);
  o.recoil += (unsigned long long)(L.eq - ch.loss_q - eq1 - wq);   // the gas's share, either sign
  const unsigned evc = L.ev - 1;
  sadd(led + (L_BIRTHS + SP_E), 1);
  sadd(led + (L_N_SPAWN_E), 1);
  Lane c;
  c.z = L.z; c.eq = wq; c.mu = (double)mu2; c.node = child_node(L.node, evc, 0);
  c.tal = 0.0; c.pid = L.pid; c.ev = 0; c.sp = SP_E; c.j = L.j; c.slot = L.slot;
  if (wq < P.ecut_q) die<F32>(P, led, c, R_CUTOFF, L_E_CUTOFF);
  else emit(port, c);
  if (ch.sout >= 0) {
    // the ion leaves with the target's velocity
    const R mi = (R)P.mass[ch.sout];
    Lane ion;
    ion.z = L.z; ion.node = child_node(L.node, evc, 1); ion.tal = 0.0; ion.pid = L.pid;
    ion.ev = 0; ion.sp = ch.sout; ion.j = L.j; ion.slot = L.slot;
    ion.eq = quant_e((double)((R)0.5 * mi * q2));
    ion.mu = q2 > (R)0 ? (double)fmin((R)1, fmax((R)-1, v2z * T::rsq(q2))) : 1.0;
    sadd(led + (L_E_IN_THERMAL), ion.eq);
    sadd(led + (L_BIRTHS + ch.sout), 1);
    sadd(led + (L_N_SPAWN_ION), 1);
    emit(port, ion);
  }
  L.eq = eq1;
  L.mu = (double)mu1;
}

// Kinematics of a charge exchange (Sec. 3.3), an ionization (Sec. 3.3
// Ionization: energy sharing, binary-encounter angles, the slow electron and
// the ion as products) or a clustering
// (Sec. 3.3 Clustering: the impactor becomes the product ion with a thermal
// target's motion) of the particle L, whose flight and channel choice are done
// (L.ev already counts this collision; w is the event's random block).
template <bool F32>
__device__ __forceinline__ void rare_kinematics(const Params& P, unsigned long long* led, Lane& L,
                                                EventOut& o, RingPort& port, int k,
                                                const unsigned long long w[4]) {
  using T = RT<F32>;
  using R = typename T::R;
  const ChanDev ch = P.ch[k];
  if (ch.kind == CHARGE_EXCHANGE) {
    charge_exchange<F32>(P, L, o.recoil);
    terminate<F32>(P, led, L, o);
    return;
  }
  const R e = T::energy(L.eq);
  if (ch.kind == IONIZATION && ch.target) {
    moving_target_ionization<F32>(P, led, L, o, port, k, w);
    terminate<F32>(P, led, L, o);
    return;
  }
  if (ch.kind == IONIZATION) {
    const long long avail = L.eq - ch.loss_q;
    const R eps = (R)P.eps_ion;
    const R wmax = (e - (R)ch.loss_ev) * (R)0.5;
    const R wsec = eps * T::tn(T::u(w[2]) * T::atn(wmax * (R)P.inv_eps_ion));
    long long wq = quant_e((double)wsec);
    if (wq > avail / 2) wq = avail / 2;
    if (wq < 0) wq = 0;
    const long long eq1 = avail - wq;
    sadd(led + (L_LOSS_IONIZ), ch.loss_q);
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
    sadd(led + (L_BIRTHS + SP_E), 1);
    sadd(led + (L_N_SPAWN_E), 1);
    Lane c;
    c.z = L.z; c.eq = wq; c.mu = (double)mu_s; c.node = child_node(L.node, evc, 0);
    c.tal = 0.0; c.pid = L.pid; c.ev = 0; c.sp = SP_E; c.j = L.j; c.slot = L.slot;
    if (wq < P.ecut_q) die<F32>(P, led, c, R_CUTOFF, L_E_CUTOFF);
    else emit(port, c);
    // ion with a thermal target's velocity (no recoil)
    if (ch.sout >= 0) {
      Lane ion;
      ion.z = L.z; ion.node = child_node(L.node, evc, 1); ion.tal = 0.0; ion.pid = L.pid;
      ion.ev = 0; ion.sp = ch.sout; ion.j = L.j; ion.slot = L.slot;
      unsigned long long wi[4];
      philox4x64_10(0ULL, ion.node, ((unsigned long long)P.pass << 8) | DOM_ION_BIRTH, 0ULL,
                    P.seed, L.pid, wi);
      thermal<F32>(P, wi, ion.eq, ion.mu);
      sadd(led + (L_E_IN_THERMAL), ion.eq);
      sadd(led + (L_BIRTHS + ch.sout), 1);
      sadd(led + (L_N_SPAWN_ION), 1);
      emit(port, ion);
    }
    L.eq = eq1;
    L.mu = (double)mu_p;
  } else {  // CLUSTERING, CLUSTERING3
    die<F32>(P, led, L, R_CLUSTER, L_E_CLUSTER);
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
    sadd(led + (L_E_IN_THERMAL), eqc);
    sadd(led + (L_BIRTHS + ch.sout), 1);
    return;
  }
  if (ch.kind == IONIZATION) terminate<F32>(P, led, L, o);
}

// The random block of the collision a parked particle chose (the event index
// before this collision was counted).
__device__ __forceinline__ void parked_block(const Params& P, const Lane& L,
                                             unsigned long long w[4]) {
  philox4x64_10((unsigned long long)(L.ev - 1), L.node,
                ((unsigned long long)P.pass << 8) | DOM_EVENT, 0ULL, P.seed, L.pid, w);
}

// Order of doubles by their bit patterns: for x >= +0.0 and any y that is not
// NaN or -0.0, x <= y exactly when bits(x) <= bits(y) as signed integers (a
// negative y has a negative pattern).  Column and position comparisons use
// it, so the segment searches take no FP64 instruction.
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
// larger and smaller of two doubles >= +0.0, by their bits
__device__ __forceinline__ double dmax_nn(double a, double b) {
  return __longlong_as_double(max(dbits(a), dbits(b)));
}
__device__ __forceinline__ double dmin_nn(double a, double b) {
  return __longlong_as_double(min(dbits(a), dbits(b)));
}

// Coefficient of channel k in this flight: sigma_k(E) interpolated at node
// interval ti, 0 at or below its loss; 1/v for an ion recombining with the
// electron field (whose per-segment value already carries sigma v).
template <bool F32>
__device__ __forceinline__ typename RT<F32>::R channel_coef(const Params& P, int k, int s,
                                                            long long eq, int ti,
                                                            typename RT<F32>::R tf,
                                                            typename RT<F32>::R inv_v) {
  using R = typename RT<F32>::R;
  const ChanDev& ch = P.ch[k];
  if (ch.kind == RECOMBINATION && s != SP_E) return inv_v;
  if (eq > ch.thr_q) {
    R a0, sl;
    RT<F32>::tab2(P, k, ti, a0, sl);
    return fma_rn(tf, sl, a0);
  }
  return (R)0;
}

// Channel choice of the per-channel path: the first channel c (selection
// order) with target < sum of the rates up to c; rates sigma_c n_j for gas
// channels and sigma_c times the channel's field at jc for field channels.
template <bool F32>
__device__ __noinline__ int select_per_channel(const Params& P, int s, long long eq, int ti,
                                               typename RT<F32>::R tf, typename RT<F32>::R inv_v,
                                               int nrec, int jc, unsigned long long w1) {
  using T = RT<F32>;
  using R = typename T::R;
  const int nsc = P.nsc[s];
  int chs = -1, last = -1;
  if (nrec == 0) {
    // gas channels only: the density of segment jc factors out
    R gas = (R)0;
    for (int c = 0; c < nsc; ++c) gas += channel_coef<F32>(P, P.sc[s][c], s, eq, ti, tf, inv_v);
    const R target = mul_rn(T::u(w1), gas);
    R cum = (R)0;
    for (int c = 0; c < nsc; ++c) {
      const R cv = channel_coef<F32>(P, P.sc[s][c], s, eq, ti, tf, inv_v);
      if (!(cv > (R)0)) continue;
      last = c;
      cum += cv;
      if (target < cum) { chs = c; break; }
    }
  } else {
    const double nj = P.nseg[jc];
    double rtot = 0.0;
    for (int c = 0; c < nsc; ++c) {
      const int kk = P.sc[s][c];
      rtot = fma_rn((double)channel_coef<F32>(P, kk, s, eq, ti, tf, inv_v),
                    field_kind(P.ch[kk].kind) ? P.frate[kk][jc] : nj, rtot);
    }
    const double target = mul_rn(u01d(w1), rtot);
    double cum = 0.0;
    for (int c = 0; c < nsc; ++c) {
      const int kk = P.sc[s][c];
      const double rk = mul_rn((double)channel_coef<F32>(P, kk, s, eq, ti, tf, inv_v),
                               field_kind(P.ch[kk].kind) ? P.frate[kk][jc] : nj);
      if (!(rk > 0.0)) continue;
      last = c;
      cum += rk;
      if (target < cum) { chs = c; break; }
    }
  }
  if (chs < 0) chs = last;                  // rounding at the top end
  return chs < 0 ? 0 : chs;
}

// Quantised time of a path of length len at 1/(|mu| v) = inv_szq / Q_T:
// round(len * inv_szq) in 2^-50 s units.
__device__ __forceinline__ unsigned long long quant_len(double len, double inv_szq) {
  return (unsigned long long)trunc_nonneg(fma_rn(len, inv_szq, 0.5));
}

template <bool F32>
__device__ void event(const Params& P, unsigned long long* led, Lane& L, EventOut& o,
                      RingPort& port) {
  using T = RT<F32>;
  using R = typename T::R;
  o.alive = true;
  o.parked = false;
  o.chan = -1;
  if (L.eq <= 0) {                 // no kinetic energy: the particle never moves
    die<F32>(P, led, L, R_STALLED, L_E_STALLED);
    o.alive = false;
    return;
  }
  const int s = L.sp;
  const R e = T::energy(L.eq);

  unsigned long long w[4];
  philox4x64_10((unsigned long long)L.ev, L.node,
                ((unsigned long long)P.pass << 8) | DOM_EVENT, 0ULL, P.seed, L.pid, w);
  const R tau = -T::lg(T::eta(w[0]));
  o.flights += 1;

  // position of ln E among the table nodes (shared by both lookups)
  const R le = T::lg(e * (R)P.inv_e_min);
  const R lx = le * (R)P.inv_h;
  int ti;
  if constexpr (F32) ti = (int)floor(lx);
  else ti = floor_or_m1(lx);                 // integer ops (below the first node: -1)
  R tf;
  int row;                                 // row of the cumulative tables (-1: none)
  if (ti < 0) { ti = 0; tf = (R)0; row = P.n_energy - 1; }          // below the first node
  else if (ti > P.n_energy - 2) { ti = P.n_energy - 2; tf = (R)1; row = -1; }
  else {
    if constexpr (F32) tf = lx - (R)ti;
    else tf = lx - i32_to_d(ti);            // the conversion on integer operations
    row = ti;
  }

  // 1/v and 1/(|mu| v) (relativistic: v = c sqrt(x (2 + x)) / (1 + x), x = E / m c^2);
  // both from one reciprocal root, and the time quantum folded into the second
  const double amu = fabs(L.mu);
  const bool still = dzero(L.mu);
  const R x = mul_rn(e, (R)P.inv_mass[s]);
  R inv_v;
  double inv_szq;                          // Q_T / (|mu| v): time units per metre along z
  if constexpr (F32) {
    inv_v = mul_rn(mul_rn((R)1 + x, (R)(1.0 / C_LIGHT)), T::rsq(mul_rn(x, (R)2 + x)));
    const float amuf = (float)amu;
    inv_szq = still ? 0.0
            : amuf > 1e-20f ? (double)mul_rn(mul_rn(inv_v, __frcp_rn(amuf)), (float)Q_T)
                            : mul_rn((double)inv_v, Q_T / amu);  // keeps FP32 in range
  } else {
    const double m2 = still ? 1.0 : mul_rn(L.mu, L.mu);
    const double base =
        mul_rn(mul_rn((R)1 + x, 1.0 / C_LIGHT), rsqrt(mul_rn(m2, mul_rn(x, (R)2 + x))));
    inv_v = still ? base : mul_rn(base, amu);
    inv_szq = mul_rn(base, Q_T);
  }

  // ---- rate coefficients of this flight ----
  const int nsc = P.nsc[s];
  const int ncg = P.ncg[s];
  // cumulative tables: the species' gas channels lead its selection order and
  // at most one channel threshold falls inside this node interval
  const int mark = ncg >= 0 && row >= 0 ? P.mixed[s * P.n_energy + row] : CUM_PER_CHANNEL;
  const bool fast = mark != CUM_PER_CHANNEL;
  // a channel that opens inside the interval: above its threshold, its own
  // interpolated cross section joins the sums from its slot xslot on
  int xslot = MAXSPCH;
  R xval = (R)0;
  if (fast && mark != CUM_PLAIN) {
    const int kx = P.sc[s][mark];
    if (L.eq > P.ch[kx].thr_q) {
      R a0, sl;
      T::tab2(P, kx, ti, a0, sl);
      xval = fma_rn(tf, sl, a0);
      xslot = mark;
    }
  }
  R gas = (R)0;
  int nrec = 0;
  double rc0 = 0.0, rc1 = 0.0;
  const double* rcol0 = P.colgas;
  const double* rcol1 = P.colgas;
  const double* rrate0 = P.nseg;
  const double* rrate1 = P.nseg;
  if (fast) {
    if (ncg > 0) {
      R a0, sl;
      T::cum2(P, s, row, ncg - 1, a0, sl);
      gas = fma_rn(tf, sl, a0) + xval;
    }
    for (int c = ncg; c < nsc; ++c) {       // field channels follow the gas channels
      const int k = P.sc[s][c];
      const R cv = channel_coef<F32>(P, k, s, L.eq, ti, tf, inv_v);
      if (nrec == 0) { rc0 = to_d(cv); rcol0 = P.fcol[k]; rrate0 = P.frate[k]; }
      else { rc1 = to_d(cv); rcol1 = P.fcol[k]; rrate1 = P.frate[k]; }
      ++nrec;
    }
  } else {
#pragma unroll 1
    for (int c = 0; c < nsc; ++c) {
      const int k = P.sc[s][c];
      const R cv = channel_coef<F32>(P, k, s, L.eq, ti, tf, inv_v);
      if (!field_kind(P.ch[k].kind)) {
        gas += cv;
      } else {
        if (nrec == 0) { rc0 = to_d(cv); rcol0 = P.fcol[k]; rrate0 = P.frate[k]; }
        else { rc1 = to_d(cv); rcol1 = P.fcol[k]; rrate1 = P.frate[k]; }
        ++nrec;
      }
    }
  }
  // energy bin of the time tally
  int b = 0;
  if (P.ntb > 1) {
    if constexpr (F32) b = (int)floor(le * (R)P.tb_scale);
    else b = floor_or_m1(le * P.tb_scale);
    b = b < 0 ? 0 : (b > P.ntb - 1 ? P.ntb - 1 : b);
  }
  const size_t trow = (size_t)P.ntb;                         // stride between z rows
  const size_t tbase = (size_t)s * (P.nz + 2) * P.ntb + b;   // (s, row 0, b)
  const size_t xbase = (size_t)s * (P.nz + 2);
  const double gasd = to_d(gas);

  // G(k) = optical-depth column of the whole rate to face k, and the rate in
  // segment j (the column tables may live in shared memory: plain loads)
  auto colsum = [&](int k) -> double {
    double g = mul_rn(gasd, P.colgas[k]);
    if (nrec > 0) g = fma_rn(rc0, rcol0[k], g);
    if (nrec > 1) g = fma_rn(rc1, rcol1[k], g);
    return g;
  };
  auto segrate = [&](int j) -> double {
    double r = mul_rn(gasd, P.nseg[j]);
    if (nrec > 0) r = fma_rn(rc0, rrate0[j], r);
    if (nrec > 1) r = fma_rn(rc1, rrate1[j], r);
    return r;
  };

  const int j0 = L.j;
  const int nz = P.nz;
  double zc;
  int jc;
  int exit_end = -1;
  // flights with gas and field channels in gas-column units: the field
  // channels' share rho = sigma_field / sigma_gas, and the field rate per
  // unit of gas density at the end segment (for the channel choice)
  bool gas_units = false;
  double rho0 = 0.0, rho1 = 0.0, rf_end = 0.0;
  if (still) {
    // no motion along z: collide in place after path tau / rate
    jc = j0;
    const double r = segrate(jc);
    if (!(r > 0.0)) {
      die<F32>(P, led, L, R_STALLED, L_E_STALLED);
      o.alive = false;
      return;
    }
    const double tfl = mul_rn((double)tau / r, (double)inv_v);
    atomicAdd(P.time_pt + tbase + (size_t)(jc + 1) * trow, quant_len(tfl, Q_T));
    if (P.track_time) L.tal += tfl;
    zc = L.z;
  } else {
    const bool up = dpos(L.mu);
    bool ex;
    if (nrec == 0) {
      // Gas only: the rate is sigma_gas n_j, so the flight ends where the gas
      // column C reaches C(z0) +- D with D = tau |mu| / sigma_gas.
      double tgt = 0.0;
      if (!dpos(gasd)) {
        ex = true;                          // no channel: straight to an end
      } else {
        double D;
        if constexpr (F32) D = (double)mul_rn(mul_rn(tau, (R)amu), __frcp_rn(gas));
        else D = mul_rn(to_d(tau), amu) / gasd;
        const double c0 = fma_rn(P.nseg[j0], L.z - P.faces[j0], P.colgas[j0]);
        tgt = up ? c0 + D : c0 - D;
        const long long tb = dbits(tgt);
        ex = up ? tb >= dbits(P.colgas[nz]) : tb <= 0;
        if (!ex) {
          // largest k with C(k) <= target, in [j0, nz) going up, [0, j0] going down
          int lo = up ? j0 : 0, hi = up ? nz : j0 + 1;
          if (P.nq > 0) {
            const float q = dtof_hint(tgt) * P.nq_over_colmax_f;
            if (q >= 0.0f && q < (float)P.nq) {
              const int qi = (int)q;
              const int a = max(lo, P.ginv[qi] - 1), bb = min(hi, P.ginv[qi + 1] + 1);
              if (a < bb && dbits(P.colgas[a]) <= tb && tb < dbits(P.colgas[bb])) {
                lo = a;
                hi = bb;
              }
            }
          }
          while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (dbits(P.colgas[mid]) <= tb) lo = mid; else hi = mid;
          }
          jc = lo;
          const double fj = P.faces[jc];
          zc = fma_rn(tgt - P.colgas[jc], P.invn[jc], fj);
          zc = dmin_nn(dmax_nn(zc, fj), P.faces[jc + 1]);
          zc = up ? dmax_nn(zc, L.z) : dmin_nn(zc, L.z);
        }
      }
    } else if (dpos(gasd)) {
      // Gas and field channels, in gas-column units: the column of the whole
      // rate over sigma_gas is G(k) = C(k) + rho0 F0(k) + rho1 F1(k), and the
      // flight ends where G reaches G(z0) +- tau |mu| / sigma_gas.  As G >= C,
      // it ends in the segment where the gas column alone reaches the target
      // or before it: the integer-compared gas search gives that segment, one
      // check of G confirms it (the fields add little rate), and otherwise the
      // search goes on before it with G.
      gas_units = true;
      const double ig = 1.0 / gasd;
      rho0 = mul_rn(rc0, ig);
      rho1 = mul_rn(rc1, ig);
      auto gcol = [&](int k) -> double {
        double g = P.colgas[k];
        if (nrec > 0) g = fma_rn(rho0, rcol0[k], g);
        if (nrec > 1) g = fma_rn(rho1, rcol1[k], g);
        return g;
      };
      auto frate = [&](int j) -> double {   // field rate per unit of gas density
        double r = 0.0;
        if (nrec > 0) r = mul_rn(rho0, rrate0[j]);
        if (nrec > 1) r = fma_rn(rho1, rrate1[j], r);
        return r;
      };
      const double c0 = fma_rn(P.nseg[j0] + frate(j0), L.z - P.faces[j0], gcol(j0));
      const double D = mul_rn(mul_rn(to_d(tau), amu), ig);
      const double tgt = up ? c0 + D : c0 - D;
      // G >= C everywhere (rho and the field columns are non-negative): a
      // target below the gas column's top is below G's top too
      ex = up ? !lt_nn(tgt, P.colgas[nz]) && !lt_nn(tgt, gcol(nz)) : !dpos(tgt);
      if (!ex) {
        const long long tb = dbits(tgt);
        int lo = up ? j0 : 0, hi = up ? nz : j0 + 1;
        if (P.nq > 0) {
          const float q = dtof_hint(tgt) * P.nq_over_colmax_f;
          if (q >= 0.0f && q < (float)P.nq) {
            const int qi = (int)q;
            const int a = max(lo, P.ginv[qi] - 1), bb = min(hi, P.ginv[qi + 1] + 1);
            if (a < bb && dbits(P.colgas[a]) <= tb && tb < dbits(P.colgas[bb])) {
              lo = a;
              hi = bb;
            }
          }
        }
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (dbits(P.colgas[mid]) <= tb) lo = mid; else hi = mid;
        }
        jc = lo;
        double gj = gcol(jc);
        if (lt_nn(tgt, gj)) {
          int l2 = up ? j0 : 0, h2 = jc;
          while (h2 - l2 > 1) {
            const int mid = (l2 + h2) >> 1;
            if (!lt_nn(tgt, gcol(mid))) l2 = mid; else h2 = mid;
          }
          jc = l2;
          gj = gcol(jc);
        }
        const double fj = P.faces[jc];
        const double gap = tgt - gj;
        const double nj = P.nseg[jc];
        rf_end = frate(jc);
        double off;
        const double eps = mul_rn(rf_end, P.invn[jc]);
        if (dpos(nj) && dabs_lt(eps, 1e-6))
          // 1 / (n + rf) = (1/n) (1 - eps + eps^2) to eps^3, eps = rf / n
          off = mul_rn(gap, mul_rn(P.invn[jc], fma_rn(-eps, 1.0 - eps, 1.0)));
        else
          off = gap / (nj + rf_end);
        zc = fj + off;
        zc = dmin_nn(dmax_nn(zc, fj), P.faces[jc + 1]);
        zc = up ? dmax_nn(zc, L.z) : dmin_nn(zc, L.z);
      }
    } else {
      // Field channels only (no gas rate): the flight inverts the column of
      // the fields, bracketed from the gas column where there is one.
      const double g0 = fma_rn(segrate(j0), L.z - P.faces[j0], colsum(j0));
      const double delta = mul_rn(to_d(tau), amu);
      const double target = up ? g0 + delta : g0 - delta;
      ex = up ? !(target < colsum(nz)) : !(target > 0.0);
      if (!ex) {
        int lo = up ? j0 : 0, hi = up ? nz : j0 + 1;
        if (gasd > 0.0 && P.nq > 0) {
          const float q = (float)target * P.nq_over_colmax_f * __frcp_rn((float)gas);
          if (q >= 0.0f && q < (float)P.nq) {
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
    }
    if (ex) {
      exit_end = up ? 1 : 0;
      zc = up ? P.L : 0.0;
      jc = up ? nz - 1 : 0;
    }
    // time in each segment crossed (Sec. 2.2): the start and end segments as
    // point adds, the full segments between as one range add; the face
    // crossings (Sec. 2.3) as one range add.  One instruction stream for a
    // flight within one segment and one across many.
    const bool same = jc == j0;
    const double fs = P.faces[up ? j0 + 1 : j0];
    const double fe = P.faces[up ? jc : jc + 1];
    const unsigned long long q0 = quant_len(fabs((same ? zc : fs) - L.z), inv_szq);
    const unsigned long long qf = quant_len(P.dz, inv_szq);
    const unsigned long long qe = quant_len(fabs(zc - fe), inv_szq);
    atomicAdd(P.time_pt + tbase + (size_t)(j0 + 1) * trow, q0);
    if (!same) {
      atomicAdd(P.time_pt + tbase + (size_t)(jc + 1) * trow, ex ? qf : qe);
      const int lo_seg = min(j0, jc), hi_seg = max(j0, jc);
      range_add(P.time_rg + tbase, lo_seg + 2, hi_seg, trow, qf);   // full segments
    }
    const int fa = up ? j0 + 1 : (ex ? 0 : jc + 1);
    const int fb = up ? (ex ? nz : jc) : j0;
    range_add((up ? P.xpos_rg : P.xneg_rg) + xbase, fa, fb, 1, 1ULL);
    if (P.track_time) L.tal = fma_rn(fabs(zc - L.z), mul_rn(inv_szq, 1.0 / Q_T), L.tal);
  }
  if (exit_end >= 0) {
    long long bin = L.eq / P.spec_bin_q;
    if (bin > P.nspec) bin = P.nspec;
    atomicAdd(P.spectrum + ((size_t)exit_end * NSP + s) * (P.nspec + 1) + bin, 1ULL);
    die<F32>(P, led, L, exit_end == 0 ? R_EXIT0 : R_EXIT1, exit_end == 0 ? L_E_EXIT0 : L_E_EXIT1);
    o.alive = false;
    return;
  }
  L.z = zc;
  L.j = jc;

  // ---- collision in segment jc: channel with probability rate_k / rate_tot ----
  L.ev += 1;
  o.colls += 1;
  int chs = -1;
  if (fast) {
    // the first channel c with target < (cumulative sigma up to c) x density;
    // a target past every gas channel falls to the field channels
    R tg;
    bool gas_part = true;
    if (nrec == 0) {
      tg = mul_rn(T::u(w[1]), gas);
    } else if (gas_units) {
      // rates per unit of gas density: gas channels n_jc (then in sigma
      // units for the cumulative tables), field channel i rho_i f_i(jc)
      const double nj = P.nseg[jc];
      const double tr = mul_rn(u01d(w[1]), nj + rf_end);
      if (lt_nn(tr, nj)) {
        tg = from_d<R>(mul_rn(mul_rn(tr, P.invn[jc]), gasd));
      } else {
        gas_part = false;
        tg = (R)0;
        double cum = nj;
        int last = -1;
        for (int c = ncg; c < nsc; ++c) {
          const int kk = P.sc[s][c];
          const double rk = mul_rn(c == ncg ? rho0 : rho1, P.frate[kk][jc]);
          if (!dpos(rk)) continue;
          last = c;
          cum += rk;
          if (lt_nn(tr, cum)) { chs = c; break; }
        }
        if (chs < 0) chs = last;
      }
    } else {
      const double nj = P.nseg[jc];
      const double target = mul_rn(u01d(w[1]), segrate(jc));
      const double gasj = mul_rn(gasd, nj);
      if (lt_nn(target, gasj)) {
        tg = from_d<R>(mul_rn(target, P.invn[jc]));
      } else {
        gas_part = false;
        tg = (R)0;
        double cum = gasj;
        int last = -1;
        for (int c = ncg; c < nsc; ++c) {
          const int kk = P.sc[s][c];
          const double rk = mul_rn(c == ncg ? rc0 : rc1, P.frate[kk][jc]);
          if (!dpos(rk)) continue;
          last = c;
          cum += rk;
          if (lt_nn(target, cum)) { chs = c; break; }
        }
        if (chs < 0) chs = last;
      }
    }
    if (gas_part) {
      for (int c = 0; c < ncg; ++c) {
        R a0, sl;
        T::cum2(P, s, row, c, a0, sl);
        if (lt_nn(tg, fma_rn(tf, sl, a0) + (c >= xslot ? xval : (R)0))) { chs = c; break; }
      }
    }
    if (chs < 0)                        // rounding at the top end
      chs = select_per_channel<F32>(P, s, L.eq, ti, tf, inv_v, nrec, jc, w[1]);
  } else {
    chs = select_per_channel<F32>(P, s, L.eq, ti, tf, inv_v, nrec, jc, w[1]);
  }
  const int k = P.sc[s][chs];
  o.chan = k;
  const ChanDev ch = P.ch[k];
  if (ch.kind == ELASTIC && ch.target) {
    moving_target_elastic<F32>(P, ch, L, w, o.recoil);
  } else if (ch.kind == ELASTIC) {
    // CM polar angle (isotropic or tabulated at the lab energy, which is the
    // impact energy for a target at rest): lab polar angle and energy transfer
    const R g = (R)P.gam[s];
    const R g2 = (R)P.gam2[s];                 // 2 g
    const R cchi = elastic_cchi<F32>(P, ch, e, T::u(w[2]));
    const R a = fma_rn(g2, cchi, fma_rn(g, g, (R)1));
    const R ra = T::rsq(a);
    const R ct = mul_rn(cchi + g, ra);
    // energy given to the target, E - E' = E 2g(1 - cos chi)/(1+g)^2
    const R de = mul_rn(mul_rn(mul_rn(e, g2), (R)1 - cchi), (R)P.inv_1pg2[s]);
    long long rq = T::quant_de(de);
    if (rq > L.eq) rq = L.eq;
    o.recoil += (unsigned long long)rq;
    L.eq -= rq;
    // sin(theta_lab) sqrt(1 - mu^2) in one root: 1 - ct^2 = (1 - cchi^2) / a
    const R cphi = T::cpi(mul_rn((R)2, T::u(w[3])));
    const R mu = from_d<R>(L.mu);
    const R ss = mul_rn(T::sq(T::max0(mul_rn(fma_rn(-cchi, cchi, (R)1), fma_rn(-mu, mu, (R)1)))),
                        ra);
    L.mu = to_d(T::clamp1(fma_rn(mu, ct, mul_rn(ss, cphi))));
  } else if (ch.kind == EXCITATION) {
    L.eq -= ch.loss_q;
    o.excit += (unsigned long long)ch.loss_q;
  } else if (ch.kind == IONIZATION || ch.kind == CLUSTERING || ch.kind == CLUSTERING3 ||
             ch.kind == CHARGE_EXCHANGE) {
    if (port.rare) {
      RareBuf* rb = port.rare;
      const int i = atomicAdd(&rb->n, 1);
      if (i < RB - rb->r) {
        rb->s[i] = L;
        rb->ch[i] = (int8_t)k;
        o.alive = false;
        o.parked = true;
        return;
      }
    }
    rare_kinematics<F32>(P, led, L, o, port, k, w);
    return;
  } else {  // RECOMBINATION
    atomicAdd(P.recomb + (size_t)ch.sout * P.nz + jc, 1ULL);
    die<F32>(P, led, L, R_RECOMB, L_E_RECOMB);
    o.alive = false;
    return;
  }
  terminate<F32>(P, led, L, o);
}

}  // namespace karl
