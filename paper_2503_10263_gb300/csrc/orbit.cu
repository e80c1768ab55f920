// orbit.cu - full-orbit transport: the Boris mover of Sec. 3.1 in a beam tube.
//
// One thread follows one particle at a time, one Boris step per loop
// iteration, so the lanes of a warp stay together on the push (the same code
// for every particle) and part only at the ends of flights.  A lane whose
// particle ends takes the next one of the generation (one atomic per
// particle).  Products (ionization secondaries and ions) are appended to the
// next generation's list with one atomic per warp; a clustering product
// replaces its ion in place.  Tallies are u64 fixed point (time, LSB
// 2^-50 s) and counts; the energy ledger is FP64.
//
// Readings (the same as the CPU oracle's): the relativistic Boris push (the
// paper's equations with u = gamma v, gamma of the half-kicked velocity in the
// rotation); the initial velocity taken as the half-step velocity; the time
// of a step booked to the z segment and radial bin of its midpoint (segment
// floor(z n_zbins / L); radial bin k for (k R / n_rbins)^2 <= x^2 + y^2 <
// ((k + 1) R / n_rbins)^2, the last bin open above), a run of
// steps in one cell rounded to the time unit once; the optical depth of a step
// the rate of its midpoint's segment times its path length; the cross
// sections those of the flight's starting energy, and with an electric field
// the flight ended, without interaction, after the step in which the kinetic
// energy leaves its bin of the time tally's energy grid (Sec. 3.1: a new
// distance is drawn when the particle leaves an energy bin); the step that
// reaches the drawn optical depth, a z end, the wall or the lifetime cap
// shortened to that fraction of its displacement (on a tie: wall, z end,
// lifetime, collision).  Directions turn in the frame of the
// unit vector towards +z normal to the old direction, so the pitch update is
// the guiding-centre one.
//
// Compiled without multiply-add contraction, so the push rounds as the
// oracle's does and histories stay matched between collisions.
#include <cooperative_groups.h>

#include "event.cuh"
#include "orbit.cuh"

namespace karl {

namespace {

enum { EV_NONE = 0, EV_WALL = 1, EV_EXIT = 2, EV_CAP = 3, EV_COLL = 4, EV_EBIN = 5 };
constexpr int DOM_REDRAW = 3;          // optical depths drawn anew after an energy-bin stop
constexpr double INV_C2 = 1.0 / (C_LIGHT * C_LIGHT);

// Comparisons of the step's tests on the bits of the doubles (integer
// operations, the same outcomes as the floating-point compares for numbers:
// a <= b for a, b >= 0 is bits(a) <= bits(b); a negative number's bits are
// negative; -0.0 counts as zero)
__device__ __forceinline__ long long bits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ bool lt0(double x) {              // x < 0
  return bits(x) < 0 && (bits(x) << 1) != 0;
}
__device__ __forceinline__ double clamp01(double f) {         // to [0, 1]
  const long long b = bits(f);
  return b < 0 ? 0.0 : (b > 0x3ff0000000000000LL ? 1.0 : f);
}

struct OPart {
  double x, y, z, ux, uy, uz, t;
  unsigned long long node, pid;
  unsigned ev;
  int sp;
};

__device__ __forceinline__ double kinetic_u(double ux, double uy, double uz, double m) {
  const double x = (ux * ux + uy * uy + uz * uz) / (C_LIGHT * C_LIGHT);
  const double g = sqrt(1.0 + x);
  return m * x / (g + 1.0);
}

__device__ __forceinline__ double proper_speed(double e, double m) {
  const double y = e / m;
  return C_LIGHT * sqrt(y * (2.0 + y));
}

// the direction at polar angle acos(ct), azimuth (cp, sp) about d (frame:
// e1 the unit vector towards +z normal to d, e2 = d x e1)
__device__ void turn(double d0, double d1, double d2, double ct, double cp, double sp,
                     double& o0, double& o1, double& o2) {
  const double s = sqrt(d0 * d0 + d1 * d1);
  double a0, a1, a2, b0, b1, b2;
  if (s > 1e-12) {
    a0 = -d2 * d0 / s; a1 = -d2 * d1 / s; a2 = s;
    b0 = d1 / s; b1 = -d0 / s; b2 = 0.0;
  } else {
    a0 = 1.0; a1 = 0.0; a2 = 0.0;
    b0 = 0.0; b1 = d2; b2 = -d1;
  }
  const double st = sqrt(fmax(0.0, 1.0 - ct * ct));
  o0 = ct * d0 + st * (cp * a0 + sp * b0);
  o1 = ct * d1 + st * (cp * a1 + sp * b1);
  o2 = ct * d2 + st * (cp * a2 + sp * b2);
}

__device__ __forceinline__ int seg_of(const Params& P, const OrbitDev& O, double z) {
  const int j = floor_or_m1(z * O.inv_dz);        // floor on the bits (negative: -1)
  return j < 0 ? 0 : (j > P.nz - 1 ? P.nz - 1 : j);
}

// radial bin of (x, y), searched from the bin b (the particle's bin, or a
// guess); the squared radii are non-negative, so they compare as integers
__device__ __forceinline__ int rbin_from(const OrbitDev& O, double x, double y, int b) {
  const long long q = __double_as_longlong(x * x + y * y);
  while (b > 0 && __double_as_longlong(__ldg(O.edge2 + b)) > q) --b;
  while (b < O.nr - 1 && __double_as_longlong(__ldg(O.edge2 + b + 1)) <= q) ++b;
  return b;
}

__device__ __forceinline__ int rbin_of(const OrbitDev& O, double x, double y) {
  int b = floor_or_m1(sqrt(x * x + y * y) * O.r_scale);
  b = b < 0 ? 0 : (b > O.nr - 1 ? O.nr - 1 : b);
  return rbin_from(O, x, y, b);
}

// cross section of channel k at energy e: linear in ln e between nodes, zero
// at or below the channel's loss, clamped to the end nodes
__device__ double sigma_e(const Params& P, int k, double e) {
  if (!(e > P.ch[k].loss_ev)) return 0.0;
  const double x = log(e * P.inv_e_min) * P.inv_h;
  int i = (int)floor(x);
  double f;
  if (i < 0) { i = 0; f = 0.0; }
  else if (i > P.n_energy - 2) { i = P.n_energy - 2; f = 1.0; }
  else { f = x - (double)i; }
  const double2 t = __ldg((const double2*)P.sig + (size_t)i * P.nch + k);
  return t.x + f * t.y;
}

// rate sums of a species at energy e: two-body channels (times n) and
// three-body clustering (times n^2)
__device__ void rate_sums(const Params& P, int s, double e, double& s1, double& s3) {
  s1 = 0.0;
  s3 = 0.0;
  for (int c = 0; c < P.nsc[s]; ++c) {
    const int k = P.sc[s][c];
    const double v = sigma_e(P, k, e);
    if (P.ch[k].kind == CLUSTERING3) s3 += v;
    else s1 += v;
  }
}

__device__ __forceinline__ void block4(const Params& P, unsigned ev, unsigned long long node,
                                       int domain, unsigned long long sub, unsigned long long pid,
                                       unsigned long long w[4]) {
  philox4x64_10((unsigned long long)ev, node, (1ULL << 8) | (unsigned long long)domain, sub,
                P.seed, pid, w);
}

// thermal product: Gamma(3/2, kT) energy, isotropic direction
__device__ void thermal3(const Params& P, unsigned ev, unsigned long long node, int domain,
                         unsigned long long pid, double& e, double& d0, double& d1, double& d2) {
  unsigned long long w[4], w2[4];
  block4(P, ev, node, domain, 0, pid, w);
  block4(P, ev, node, domain, 1, pid, w2);
  const double TWO_PI = 6.283185307179586476925286766559;
  const double c = cos(TWO_PI * u01d(w[2]));
  e = P.kT * (-log(eta01d(w[0])) - log(eta01d(w[1])) * c * c);
  double mu = 2.0 * u01d(w[3]);
  mu -= 1.0;
  const double st = sqrt(fmax(0.0, 1.0 - mu * mu));
  const double ph = TWO_PI * u01d(w2[0]);
  d0 = st * cos(ph);
  d1 = st * sin(ph);
  d2 = mu;
}

__device__ __forceinline__ void set_u(const Params& P, OPart& Q, double e, double d0, double d1,
                                      double d2) {
  const double ps = proper_speed(e, P.mass[Q.sp]);
  Q.ux = ps * d0;
  Q.uy = ps * d1;
  Q.uz = ps * d2;
}

// products go to the next generation's list, one atomic per warp
__device__ void push_product(const OrbitDev& O, const OPart& Q) {
  namespace cg = cooperative_groups;
  cg::coalesced_group g = cg::coalesced_threads();
  unsigned long long base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(O.counters + 1, (unsigned long long)g.size());
  base = g.shfl(base, 0);
  const unsigned long long i = base + g.thread_rank();
  if (i >= O.out_cap) {
    atomicMax(O.error, ERR_CAPACITY);
    return;
  }
  O.out.x[i] = Q.x; O.out.y[i] = Q.y; O.out.z[i] = Q.z;
  O.out.ux[i] = Q.ux; O.out.uy[i] = Q.uy; O.out.uz[i] = Q.uz;
  O.out.node[i] = Q.node; O.out.pid[i] = Q.pid; O.out.sp[i] = (uint8_t)Q.sp;
}

__device__ __forceinline__ void die(const Params& P, const OrbitDev& O, const OPart& Q, int reason,
                                    int eslot, double e) {
  atomicAdd(O.ledger + OB_DEATHS + Q.sp * NREASON + reason, 1ULL);
  atomicAdd(O.energy + eslot, e);
  const long long i = (long long)Q.pid - P.pid_offset;
  if (O.per_primary && Q.ev > 0) atomicAdd(O.per_primary + i, (unsigned long long)Q.ev);
  if (O.end_state && Q.node == 0) {
    double* es = O.end_state + 8 * i;
    es[0] = Q.x; es[1] = Q.y; es[2] = Q.z;
    es[3] = kinetic_u(Q.ux, Q.uy, Q.uz, P.mass[Q.sp]);
    es[4] = Q.ux; es[5] = Q.uy; es[6] = Q.uz; es[7] = Q.t;
  }
}

__device__ __forceinline__ void flush_run(const Params& P, const OrbitDev& O, int s, int cj,
                                          int cr, unsigned long long cn, double f_last,
                                          double dt) {
  if (cj < 0) return;
  const double t = (double)cn * dt + f_last * dt;
  const unsigned long long q = (unsigned long long)(t * Q_T + 0.5);
  atomicAdd(O.time_z + (size_t)s * P.nz + cj, q);
  atomicAdd(O.time_r + (size_t)s * O.nr + cr, q);
}

// crossings of z faces and radial bin boundaries by a step from segment ja,
// radial bin ra to segment jb, radial bin rb
__device__ void crossings(const Params& P, const OrbitDev& O, int s, int ja, int ra, int jb,
                          int rb) {
  const int nz = P.nz, nr = O.nr;
  for (int k = ja + 1; k <= jb; ++k) atomicAdd(O.xpos + (size_t)s * (nz + 1) + k, 1ULL);
  for (int k = jb + 1; k <= ja; ++k) atomicAdd(O.xneg + (size_t)s * (nz + 1) + k, 1ULL);
  for (int k = ra + 1; k <= rb; ++k) atomicAdd(O.rout + (size_t)s * (nr + 1) + k, 1ULL);
  for (int k = rb + 1; k <= ra; ++k) atomicAdd(O.rin + (size_t)s * (nr + 1) + k, 1ULL);
}

struct Flight {
  double tau, acc, e0, s1, s3;
  double u2lo, u2hi;               // the flight's energy bin as bounds on u^2
  unsigned long long step;
  int cj, cr;                      // cell of the current run of steps
  unsigned long long cn;
  int js, rs;                      // segment and radial bin of the particle
  unsigned redraw;                 // energy-bin stops since the last event
  unsigned long long w1, w2, w3;   // uniforms of the collision
};

// Start a flight; false if the particle cannot move (stalled, ended here).
__device__ bool start_flight(const Params& P, const OrbitDev& O, OPart& Q, Flight& F) {
  const double m = P.mass[Q.sp];
  F.e0 = kinetic_u(Q.ux, Q.uy, Q.uz, m);
  if (!(F.e0 > 0.0)) {
    die(P, O, Q, OR_STALLED, OE_STALLED, F.e0);
    return false;
  }
  unsigned long long w[4];
  block4(P, Q.ev, Q.node, DOM_EVENT, 0, Q.pid, w);
  F.tau = -log(eta01d(w[0]));
  if (F.redraw > 0) {
    unsigned long long wr[4];
    block4(P, Q.ev, Q.node, DOM_REDRAW, F.redraw, Q.pid, wr);
    F.tau = -log(eta01d(wr[0]));
  }
  F.w1 = w[1]; F.w2 = w[2]; F.w3 = w[3];
  F.acc = 0.0;
  rate_sums(P, Q.sp, F.e0, F.s1, F.s3);
  F.u2lo = -1.0;
  F.u2hi = INFINITY;
  if (O.fields) {
    const int ntb = P.ntb;
    int b = 0;
    if (ntb > 1) {
      const double x = log(F.e0 / P.e_min) / log(O.e_max / P.e_min) * (double)ntb;
      b = (int)floor(x);
      b = b < 0 ? 0 : (b > ntb - 1 ? ntb - 1 : b);
    }
    const double* edge = O.u2edge + (size_t)Q.sp * (ntb + 1);
    if (b > 0) F.u2lo = edge[b];
    if (b < ntb - 1) F.u2hi = edge[b + 1];
  }
  F.step = 0;
  F.cj = -1; F.cr = -1; F.cn = 0;
  F.js = seg_of(P, O, Q.z);
  F.rs = rbin_of(O, Q.x, Q.y);
  atomicAdd(O.ledger + OB_N_FLIGHT, 1ULL);
  return true;
}

// The collision at the end of a flight (Sec. 3.3 kinematics in three
// dimensions).  Returns false if the particle ended.
__device__ bool collide(const Params& P, const OrbitDev& O, OPart& Q, Flight& F) {
  const double TWO_PI = 6.283185307179586476925286766559;
  const int s = Q.sp;
  const double m = P.mass[s];
  const int j = seg_of(P, O, Q.z);
  Q.ev += 1;
  atomicAdd(O.ledger + OB_N_COLL, 1ULL);
  const double ec = kinetic_u(Q.ux, Q.uy, Q.uz, m);
  const double esig = F.e0;
  const double n = P.nseg[j];
  // channel k with probability rate_k / rate_tot (table order)
  double rtot = 0.0;
  for (int c = 0; c < P.nsc[s]; ++c) {
    const int k = P.sc[s][c];
    const double sk = sigma_e(P, k, esig);
    rtot += P.ch[k].kind == CLUSTERING3 ? sk * (n * n) : sk * n;
  }
  const double target = u01d(F.w1) * rtot;
  int ch = -1, last = -1;
  double cum = 0.0;
  for (int c = 0; c < P.nsc[s]; ++c) {
    const int k = P.sc[s][c];
    const double sk = sigma_e(P, k, esig);
    const double rk = P.ch[k].kind == CLUSTERING3 ? sk * (n * n) : sk * n;
    if (!(rk > 0.0)) continue;
    last = k;
    cum += rk;
    if (target < cum) { ch = k; break; }
  }
  if (ch < 0) ch = last;
  if (ch < 0) {                                       // no open channel: cannot happen
    die(P, O, Q, OR_STALLED, OE_STALLED, ec);
    return false;
  }
  atomicAdd(O.chan + ch, 1ULL);
  const ChanDev& cd = P.ch[ch];
  const double pu = sqrt(Q.ux * Q.ux + Q.uy * Q.uy + Q.uz * Q.uz);
  const double d0 = Q.ux / pu, d1 = Q.uy / pu, d2 = Q.uz / pu;
  const double ph = TWO_PI * u01d(F.w3);
  const double cph = cos(ph), sph = sin(ph);
  const unsigned evc = Q.ev - 1;
  F.redraw = 0;
  double enew = ec;
  if (cd.kind == ELASTIC) {
    const double g = P.gam[s];
    const double cchi = elastic_cchi<false>(P, cd, ec, u01d(F.w2));
    const double a = 1.0 + 2.0 * g * cchi + g * g;
    const double ct = (cchi + g) / sqrt(a);
    const double loss = ec * 2.0 * g * (1.0 - cchi) / ((1.0 + g) * (1.0 + g));
    enew = ec - loss;
    atomicAdd(O.energy + OE_RECOIL, loss);
    double o0, o1, o2;
    turn(d0, d1, d2, ct, cph, sph, o0, o1, o2);
    set_u(P, Q, enew, o0, o1, o2);
  } else if (cd.kind == EXCITATION) {
    enew = ec - cd.loss_ev;
    atomicAdd(O.energy + OE_LOSS_EXCIT, cd.loss_ev);
    set_u(P, Q, enew, d0, d1, d2);
  } else if (cd.kind == IONIZATION) {
    const double ion_e = cd.loss_ev;
    const double avail = ec - ion_e;
    const double eps = P.eps_ion;
    double wsec = eps * tan(u01d(F.w2) * atan(0.5 * avail / eps));
    if (wsec > 0.5 * avail) wsec = 0.5 * avail;
    if (wsec < 0.0) wsec = 0.0;
    enew = avail - wsec;
    atomicAdd(O.energy + OE_LOSS_IONIZ, ion_e);
    const double cp = avail > 0.0 ? sqrt(enew / avail) : 1.0;
    const double sp = avail > 0.0 ? sqrt(wsec / avail) : 0.0;
    double o0, o1, o2, q0, q1, q2;
    turn(d0, d1, d2, cp, cph, sph, o0, o1, o2);
    turn(d0, d1, d2, sp, -cph, -sph, q0, q1, q2);     // secondary azimuth = primary's - pi
    set_u(P, Q, enew, o0, o1, o2);
    OPart S;
    S.x = Q.x; S.y = Q.y; S.z = Q.z; S.t = 0.0; S.ev = 0; S.sp = SP_E;
    S.node = child_node(Q.node, evc, 0);
    S.pid = Q.pid;
    set_u(P, S, wsec, q0, q1, q2);
    atomicAdd(O.ledger + OB_BIRTHS + SP_E, 1ULL);
    atomicAdd(O.ledger + OB_N_SPAWN_E, 1ULL);
    if (wsec < O.e_cut) die(P, O, S, OR_CUTOFF, OE_CUTOFF, wsec);
    else push_product(O, S);
    if (cd.sout >= 0) {
      OPart I;
      I.x = Q.x; I.y = Q.y; I.z = Q.z; I.t = 0.0; I.ev = 0; I.sp = cd.sout;
      I.node = child_node(Q.node, evc, 1);
      I.pid = Q.pid;
      double ei, i0, i1, i2;
      thermal3(P, 0, I.node, DOM_ION_BIRTH, I.pid, ei, i0, i1, i2);
      set_u(P, I, ei, i0, i1, i2);
      atomicAdd(O.energy + OE_IN_THERMAL, ei);
      atomicAdd(O.ledger + OB_BIRTHS + cd.sout, 1ULL);
      atomicAdd(O.ledger + OB_N_SPAWN_ION, 1ULL);
      push_product(O, I);
    }
  } else {                                           // clustering: the product replaces the ion
    die(P, O, Q, OR_CLUSTER, OE_CLUSTER, ec);
    OPart C;
    C.x = Q.x; C.y = Q.y; C.z = Q.z; C.t = 0.0; C.ev = 0; C.sp = cd.sout;
    C.node = child_node(Q.node, evc, 2);
    C.pid = Q.pid;
    double ecl, c0, c1, c2;
    thermal3(P, evc, Q.node, DOM_CLUSTER, Q.pid, ecl, c0, c1, c2);
    set_u(P, C, ecl, c0, c1, c2);
    atomicAdd(O.energy + OE_IN_THERMAL, ecl);
    atomicAdd(O.ledger + OB_BIRTHS + C.sp, 1ULL);
    Q = C;
    return true;
  }
  // terminator (Sec. 3.2)
  if (s == SP_E && enew < O.e_cut) { die(P, O, Q, OR_CUTOFF, OE_CUTOFF, enew); return false; }
  if (Q.ev >= P.max_coll) { die(P, O, Q, OR_CAP_COLL, OE_CAP, enew); return false; }
  if (Q.t >= P.max_life) { die(P, O, Q, OR_CAP_TIME, OE_CAP, enew); return false; }
  return true;
}

// Load particle i of the generation; false if it ended at birth.
__device__ bool load(const Params& P, const OrbitDev& O, long long i, OPart& Q) {
  Q.t = 0.0;
  Q.ev = 0;
  if (O.from_primaries) {
    Q.x = O.px[i]; Q.y = O.py[i]; Q.z = O.pz[i];
    Q.sp = O.psp[i];
    Q.node = 0;
    Q.pid = (unsigned long long)(P.pid_offset + i);
    const double e = O.pe[i], mu = O.pmu[i], ph = O.pphi[i];
    const double st = sqrt(fmax(0.0, 1.0 - mu * mu));
    set_u(P, Q, e, st * cos(ph), st * sin(ph), mu);
    atomicAdd(O.energy + OE_IN_PRIMARY, e);
    atomicAdd(O.ledger + OB_BIRTHS + Q.sp, 1ULL);
    if (Q.sp == SP_E && e < O.e_cut) {
      die(P, O, Q, OR_CUTOFF, OE_CUTOFF, e);
      return false;
    }
    return true;
  }
  Q.x = O.in.x[i]; Q.y = O.in.y[i]; Q.z = O.in.z[i];
  Q.ux = O.in.ux[i]; Q.uy = O.in.uy[i]; Q.uz = O.in.uz[i];
  Q.node = O.in.node[i];
  Q.pid = O.in.pid[i];
  Q.sp = O.in.sp[i];
  return true;
}

__global__ void __launch_bounds__(256) orbit_kernel(const Params P, const OrbitDev O) {
  const double L = P.L;
  bool live = false;
  OPart Q;
  Flight F;
  unsigned long long steps = 0;
  const unsigned long long t_end = globaltimer_ns() + O.timeout_ns;
  for (unsigned long long it = 0;; ++it) {
    if ((it & 1023) == 0) {
      if (*(volatile int*)O.error != ERR_NONE) break;
      if (O.cancel && *O.cancel) { atomicMax(O.error, ERR_CANCELLED); break; }
      if (globaltimer_ns() > t_end) { atomicMax(O.error, ERR_TIMEOUT); break; }
    }
    if (!live) {
      const long long i = (long long)atomicAdd(O.counters, 1ULL);
      if (i >= O.n_in) break;
      if (!load(P, O, i, Q)) continue;
      F.redraw = 0;
      live = start_flight(P, O, Q, F);
      continue;
    }
    const int s = Q.sp;
    const double m = P.mass[s];
    const double dt = O.dt[s];
    const double h = O.h[s];
    if (F.step >= O.max_steps) {
      flush_run(P, O, s, F.cj, F.cr, F.cn, 0.0, dt);
      const double e = kinetic_u(Q.ux, Q.uy, Q.uz, m);
      atomicAdd(O.energy + OE_FIELD_WORK, e - F.e0);
      die(P, O, Q, OR_STALLED, OE_STALLED, e);
      live = false;
      continue;
    }
    F.step += 1;
    steps += 1;
    // Boris push: half electric kick, magnetic rotation, half kick
    const double ex = O.er * Q.x, ey = O.er * Q.y, ez = O.ez ? O.ez[F.js] : 0.0;
    const double umx = Q.ux + h * ex, umy = Q.uy + h * ey, umz = Q.uz + h * ez;
    const double gm = sqrt(1.0 + (umx * umx + umy * umy + umz * umz) * INV_C2);
    const double t = h * O.bz / gm;
    const double sf = 2.0 * t / (1.0 + t * t);
    const double upx = umx + umy * t, upy = umy - umx * t;
    const double unx = umx + upy * sf + h * ex;
    const double uny = umy - upx * sf + h * ey;
    const double unz = umz + h * ez;
    const double u2n = unx * unx + uny * uny + unz * unz;
    const double gn = sqrt(1.0 + u2n * INV_C2);
    const double sc = dt / gn;
    const double dx = unx * sc, dy = uny * sc, dz = unz * sc;
    const double ds = sqrt(dx * dx + dy * dy + dz * dz);
    const int jm = seg_of(P, O, Q.z + 0.5 * dz);
    const double nm = P.nseg[jm];
    const double dtau = (F.s1 * nm + F.s3 * (nm * nm)) * ds;
    // the first of wall, z end, lifetime cap and collision within the step
    double fb = 1.0;
    int event = EV_NONE, end = -1;
    const double xn = Q.x + dx, yn = Q.y + dy, zn = Q.z + dz;
    if (bits(xn * xn + yn * yn) > bits(O.R2)) {
      const double a = dx * dx + dy * dy;
      const double b = Q.x * dx + Q.y * dy;
      const double c = Q.x * Q.x + Q.y * Q.y - O.R2;
      const double disc = sqrt(fmax(0.0, b * b - a * c));
      double f = dpos(b) ? -c / (b + disc) : (disc - b) / a;
      f = clamp01(f);
      if (f <= fb) { fb = f; event = EV_WALL; }
    }
    const bool below = lt0(zn);
    if (below || bits(zn) > bits(L)) {
      double f = below ? -Q.z / dz : (L - Q.z) / dz;
      f = clamp01(f);
      if (event == EV_NONE ? f <= fb : f < fb) { fb = f; event = EV_EXIT; end = below ? 0 : 1; }
    }
    if (bits(Q.t + dt) >= bits(P.max_life)) {
      const double f = clamp01((P.max_life - Q.t) / dt);
      if (event == EV_NONE ? f <= fb : f < fb) { fb = f; event = EV_CAP; }
    }
    if (dpos(dtau) && bits(F.acc + dtau) >= bits(F.tau)) {
      const double f = clamp01((F.tau - F.acc) / dtau);
      if (event == EV_NONE ? f <= fb : f < fb) { fb = f; event = EV_COLL; }
    }
    if (event == EV_NONE && (bits(u2n) < bits(F.u2lo) || bits(u2n) >= bits(F.u2hi)))
      event = EV_EBIN;
    if (event == EV_NONE || event == EV_EBIN) {
      const int mr = rbin_from(O, Q.x + 0.5 * dx, Q.y + 0.5 * dy, F.rs);
      if (jm == F.cj && mr == F.cr) {
        F.cn += 1;
      } else {
        flush_run(P, O, s, F.cj, F.cr, F.cn, 0.0, dt);
        F.cj = jm; F.cr = mr; F.cn = 1;
      }
      const int jb = seg_of(P, O, zn), rb = rbin_from(O, xn, yn, F.rs);
      if (jb != F.js || rb != F.rs) {
        crossings(P, O, s, F.js, F.rs, jb, rb);
        F.js = jb;
        F.rs = rb;
      }
      Q.x = xn; Q.y = yn; Q.z = zn;
      Q.t += dt;
      F.acc += dtau;
      Q.ux = unx; Q.uy = uny; Q.uz = unz;
      if (event == EV_NONE) continue;
      // left the energy bin: the run's time, then a new flight
      flush_run(P, O, s, F.cj, F.cr, F.cn, 0.0, dt);
      atomicAdd(O.energy + OE_FIELD_WORK, kinetic_u(Q.ux, Q.uy, Q.uz, m) - F.e0);
      F.redraw += 1;
      live = start_flight(P, O, Q, F);
      continue;
    }
    // the shortened last step of the flight
    const double px = fb * dx, py = fb * dy, pz = fb * dz;
    const int mj = seg_of(P, O, Q.z + 0.5 * pz), mr = rbin_of(O, Q.x + 0.5 * px, Q.y + 0.5 * py);
    if (mj == F.cj && mr == F.cr) {
      flush_run(P, O, s, F.cj, F.cr, F.cn, fb, dt);
    } else {
      flush_run(P, O, s, F.cj, F.cr, F.cn, 0.0, dt);
      flush_run(P, O, s, mj, mr, 0, fb, dt);
    }
    const double bx = Q.x + px, by = Q.y + py;
    const double bz = event == EV_EXIT ? (end == 0 ? 0.0 : L) : Q.z + pz;
    crossings(P, O, s, F.js, F.rs, seg_of(P, O, bz), rbin_of(O, bx, by));
    Q.x = bx; Q.y = by; Q.z = bz;
    Q.t = event == EV_CAP ? P.max_life : Q.t + fb * dt;
    Q.ux = unx; Q.uy = uny; Q.uz = unz;
    const double e1 = kinetic_u(Q.ux, Q.uy, Q.uz, m);
    atomicAdd(O.energy + OE_FIELD_WORK, e1 - F.e0);
    if (event == EV_WALL) {
      atomicAdd(O.wall + (size_t)s * P.nz + seg_of(P, O, Q.z), 1ULL);
      const int ra = rbin_of(O, Q.x, Q.y);
      for (int k = ra + 1; k <= O.nr; ++k) atomicAdd(O.rout + (size_t)s * (O.nr + 1) + k, 1ULL);
      die(P, O, Q, OR_WALL, OE_WALL, e1);
      live = false;
      continue;
    }
    if (event == EV_EXIT) {
      if (end == 1) atomicAdd(O.xpos + (size_t)s * (P.nz + 1) + P.nz, 1ULL);
      else atomicAdd(O.xneg + (size_t)s * (P.nz + 1), 1ULL);
      const double xb = floor(e1 / O.spec_bin);
      const long long bin = xb < 0.0 ? 0 : (xb > (double)P.nspec ? P.nspec : (long long)xb);
      atomicAdd(O.spectrum + ((size_t)end * NSP + s) * (P.nspec + 1) + bin, 1ULL);
      die(P, O, Q, end == 0 ? OR_EXIT0 : OR_EXIT1, end == 0 ? OE_EXIT0 : OE_EXIT1, e1);
      live = false;
      continue;
    }
    if (event == EV_CAP) {
      die(P, O, Q, OR_CAP_TIME, OE_CAP, e1);
      live = false;
      continue;
    }
    live = collide(P, O, Q, F) && start_flight(P, O, Q, F);
  }
  if (steps) atomicAdd(O.ledger + OB_N_STEP, steps);
}

}  // namespace

cudaError_t launch_orbit(const Params& P, const OrbitDev& O, int grid, int block,
                         cudaStream_t st) {
  orbit_kernel<<<grid, block, 0, st>>>(P, O);
  return cudaGetLastError();
}

cudaError_t orbit_occupancy(int block, int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, orbit_kernel, block, 0);
}

}  // namespace karl
