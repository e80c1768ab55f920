// karl_device.cuh - device-side types and helpers of the KARL transport path.
//
// Random numbers: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11), keyed by (seed, primary id) with the
// counter (event index, lineage id, pass << 8 | domain, sub-index).  Streams
// are therefore independent of scheduling order, batch mix and grid shape.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace karl {

constexpr int NSP = 4;            // e-, T2+, T3+, T+
constexpr int MAXCH = 16;         // channels in the tables
constexpr int MAXSPCH = 10;       // active channels of one species
constexpr int LEDGER = 64;
constexpr int NREASON = 8;

enum { ELASTIC = 0, IONIZATION = 1, EXCITATION = 2, CLUSTERING = 3, RECOMBINATION = 4,
       CHARGE_EXCHANGE = 5, CLUSTERING3 = 6 };

// channels whose rate per unit path follows a field other than the gas density
// n(z): recombination (the partner's target field) and three-body clustering
// (n(z)^2); their flights invert that field's column beside the gas column
__host__ __device__ __forceinline__ bool field_kind(int kind) {
  return kind == RECOMBINATION || kind == CLUSTERING3;
}
enum { SP_E = 0 };
// Marks of the cumulative cross-section tables, per species and node
// interval: the interval needs nothing more (CUM_PLAIN), one of its gas
// channels opens inside it (the channel's slot: above the channel's threshold
// its own interpolated cross section is added to the cumulative sums from its
// slot on), or the per-channel path (CUM_PER_CHANNEL).
constexpr unsigned char CUM_PLAIN = 255;
constexpr unsigned char CUM_PER_CHANNEL = 254;
enum { R_EXIT0 = 0, R_EXIT1 = 1, R_CUTOFF = 2, R_CAP_COLL = 3, R_CAP_TIME = 4,
       R_RECOMB = 5, R_CLUSTER = 6, R_STALLED = 7 };
enum { L_E_IN_PRIMARY = 0, L_E_IN_THERMAL = 1, L_E_EXIT0 = 2, L_E_EXIT1 = 3, L_E_CUTOFF = 4,
       L_E_CAP = 5, L_E_RECOMB = 6, L_E_CLUSTER = 7, L_LOSS_IONIZ = 8, L_LOSS_EXCIT = 9,
       L_LOSS_RECOIL = 10, L_E_STALLED = 11, L_BIRTHS = 12, L_DEATHS = 16, L_N_COLL = 48,
       L_N_FLIGHT = 49, L_N_SPAWN_E = 50, L_N_SPAWN_ION = 51, L_N_COLL_ALL = 52,
       L_N_FLIGHT_ALL = 53 };
enum { DOM_EVENT = 0, DOM_ION_BIRTH = 1, DOM_CLUSTER = 2, DOM_TARGET = 4 };
enum { ERR_NONE = 0, ERR_TIMEOUT = 4, ERR_CAPACITY = 6, ERR_CANCELLED = 7 };

struct ChanDev {
  int32_t kind, sin, sout, target;   // target: 0 at rest, 1 moving (elastic, ionization)
  int32_t ang, pad;        // angle-table set of an elastic channel, -1 isotropic
  long long loss_q;        // loss in 2^-24 eV units (floor)
  long long thr_q;         // channel open iff eq > thr_q  (E > loss_ev exactly)
  double loss_ev;
};

// Everything one pass of the transport kernel reads.  Passed by value.
struct Params {
  // geometry and gas (Sec. 2.2 segmentation)
  int nz;
  double L, dz;
  const double* nseg;      // [nz] gas density per segment
  const double* colgas;    // [nz+1] column to each face, sum_{i<k} n_i dz
  const double* faces;     // [nz+1] face positions k*dz (face nz = L exactly)
  const int* ginv;         // [nq+1] largest face k with colgas[k] <= q * colmax / nq
  const double* invn;      // [nz] 1 / n_j (0 in a segment without gas)
  int nq;
  double nq_over_colmax;   // nq / colgas[nz] (0 if the column is empty)
  float nq_over_colmax_f;  // same in FP32 (search hints only)
  // recombination target fields of pass 2, per channel (NULL if unused)
  const double* frate[MAXCH];   // [nz] partner field per segment
  const double* fcol[MAXCH];    // [nz+1] its column to each face
  // cross sections
  int n_energy;
  double e_min, inv_e_min, log_ratio_h, inv_h;   // h = ln(e_max/e_min)/(n-1)
  const double* sig;            // [n_energy][nch], the channels of one node together
  const float* sigf;            // same, FP32
  // cumulative cross sections of each species' leading gas channels over the
  // channels open in a node interval, pairs (value, slope) at
  // [cum_off[s] + i * ncg[s] + c]; intervals holding a channel threshold are
  // marked in mixed[s * n_energy + i] (per-channel path there)
  const double* cum;
  const float* cumf;
  const unsigned char* mixed;
  int ncg[NSP];                 // leading gas channels of the species (0: per-channel path)
  int cum_off[NSP];
  int nch;
  ChanDev ch[MAXCH];
  // scattering-angle tables of elastic channels (Sec. 3.3 Elastic): per set
  // and impact-energy bin, the pdf of cos chi on n_mu even points over
  // [-1, 1] and its cumulative integral (trapezoids: exact for the
  // piecewise-linear pdf); NULL when every channel is isotropic
  int ang_nb, ang_nmu;
  double ang_h, ang_inv_h;      // point spacing 2 / (n_mu - 1) and its inverse
  const double* ang_pdf;        // [sets][bins][n_mu]
  const double* ang_cum;        // [sets][bins][n_mu], starts at 0
  const float* ang_pdff;        // FP32 copies
  const float* ang_cumf;
  double ang_inv_lo[MAXCH];     // 1 / e_min of each set
  double ang_scale[MAXCH];      // n_bins / ln(e_max / e_min)
  double ang_thr[MAXCH];        // isotropic below this impact energy
  int nsc[NSP];
  int8_t sc[NSP][MAXSPCH];      // active channels per species, in selection order
  // species and targets
  double mass[NSP];
  double inv_mass[NSP];
  double gam[NSP];              // m / M_target
  double gam2[NSP];             // 2 m / M_target
  double inv_1pg2[NSP];         // 1 / (1 + m/M)^2
  double target_mass, eps_ion, inv_eps_ion, kT;
  double drift_c;               // gas drift along +z in units of c (moving targets)
  double target_a;              // sqrt(kT / target mass): thermal velocity component, units of c
  long long ecut_q;
  unsigned max_coll;
  double max_life;
  int track_time;               // a lifetime cap is set: accumulate time alive
  int ntb;
  double tb_scale;              // ntb / ln(e_max/e_min)
  int nspec;
  long long spec_bin_q;
  // random streams
  unsigned long long seed;
  int pass;
  long long pid_offset;
  // primaries (device)
  long long n_prim;
  const double* pz;
  const double* pe;
  const double* pmu;
  const uint8_t* psp;
  // raw tallies (device)
  unsigned long long* spectrum;   // [2][4][nspec+1]
  unsigned long long* time_pt;    // [4][nz+2][ntb] point adds
  unsigned long long* time_rg;    // [4][nz+2][ntb] range adds (difference form)
  unsigned long long* xpos_rg;    // [4][nz+2] face crossings +z (difference form)
  unsigned long long* xneg_rg;    // [4][nz+2] face crossings -z (difference form)
  unsigned long long* recomb;     // [4][nz]
  unsigned long long* ledger;     // [64]
  unsigned long long* chan_count; // [nch]
  unsigned long long* per_primary;// [n_prim] or NULL
};

// Particle ring (structure of arrays) shared by all warps of a pass.
struct Ring {
  double* z;
  long long* eq;
  double* mu;
  unsigned long long* node;
  double* tal;
  unsigned long long* pid;
  unsigned* ev;
  unsigned* sj;                 // segment index << 8 | species
  unsigned long long* seq;      // per-cell sequence number (bounded MPMC ring)
  unsigned long long cap, mask;
};

// Work counters of one pass.  The four hot counters sit on separate 128-byte
// lines so their atomics do not serialise on one L2 line.
struct Control {
  unsigned long long head;      // next ring position to consume
  char pad0[120];
  unsigned long long tail;      // next ring position to produce
  char pad1[120];
  unsigned long long prim_next; // next primary index
  char pad2[120];
  long long active;             // particles held by lanes (current + lane stacks)
  char pad3[120];
  int error;
  int abort;
  unsigned long long particles; // particles started (primaries + products)
  unsigned long long idle_iters;      // warp iterations without a particle
  unsigned long long busy_iters;      // warp iterations with at least one
  unsigned long long busy_lane_iters; // lanes holding a particle, summed over busy iterations
  unsigned long long spilled;         // products sent to the shared ring
  // device clock (ns): first block started, last primary claimed, last warp left
  unsigned long long t_start, t_claimed, t_end;
};

// ------------------------------------------------------------------------
// Philox4x64-10

__device__ __forceinline__ void philox4x64_10(unsigned long long c0, unsigned long long c1,
                                              unsigned long long c2, unsigned long long c3,
                                              unsigned long long k0, unsigned long long k1,
                                              unsigned long long out[4]) {
  const unsigned long long M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const unsigned long long W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    unsigned long long hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
    unsigned long long hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
    unsigned long long n0 = hi1 ^ c1 ^ k0;
    unsigned long long n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += W0; k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// SplitMix64 output function (Steele, Lea, Flood 2014): lineage ids of products
__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  unsigned long long z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
__device__ __forceinline__ unsigned long long child_node(unsigned long long parent, unsigned ev,
                                                         unsigned slot) {
  return mix64(mix64(parent) ^ (((unsigned long long)ev << 2) | slot));
}

// Integer-to-double conversions run on GB300's FP64 pipe (16 SM-cycles a
// warp instruction, like an FP64 fma); these build the same values from the
// bits with integer operations.
// m 2^-k for 0 <= m < 2^53 (exact): the leading bit p of m sets the exponent,
// the bits below it the significand
__device__ __forceinline__ double u53_scaled(unsigned long long m, int k) {
  if (m == 0) return 0.0;
  const int p = 63 - __clzll((long long)m);
  return __longlong_as_double(((long long)(1023 + p - k) << 52) |
                              (long long)((m << (52 - p)) & 0x000fffffffffffffULL));
}
// (double)k for |k| < 2^31
__device__ __forceinline__ double i32_to_d(int k) {
  const double d = u53_scaled((unsigned long long)(k < 0 ? -(long long)k : (long long)k), 0);
  return k < 0 ? __longlong_as_double(__double_as_longlong(d) | (long long)0x8000000000000000ULL) : d;
}
// ln x for positive normal x, table-driven (P. T. P. Tang, "Table-driven
// implementation of the logarithm function in IEEE floating-point
// arithmetic", ACM TOMS 16, 1990): x = 2^k m with m in [1, 2) in one of 256
// cells of centre c_j, m = c_j (1 + r), |r| <= 1/512, and
// ln x = k ln 2 + ln c_j + ln(1 + r), the last by its Taylor series to r^6
// (truncation below 3e-20).  Absolute error about 2e-16 (the rounding of
// 1/c_j carried into r) plus the rounding of k ln 2: the accuracy the flight
// optical depth and the table position need, in about 9 FP64 operations.
__device__ const double2 karl_log_cells[256] = {
#include "log_table.inc"
};

__device__ __forceinline__ double log_tab(double x) {
  const long long bits = __double_as_longlong(x);
  const int k = (int)((bits >> 52) & 0x7ff) - 1023;
  const int j = (int)((bits >> 44) & 0xff);
  const double m = __longlong_as_double((bits & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
  const double2 c = __ldg(karl_log_cells + j);            // (ln c_j, 1 / c_j)
  const double r = __fma_rn(m, c.y, -1.0);
  // Horner's form with explicit fused multiply-adds (the same bits in every kernel)
  double t = __fma_rn(r, -1.0 / 6.0, 0.2);
  t = __fma_rn(r, t, -0.25);
  t = __fma_rn(r, t, 1.0 / 3.0);
  t = __fma_rn(r, t, -0.5);
  t = __fma_rn(r, t, 1.0);
  return __fma_rn(i32_to_d(k), 0.69314718055994530942, __dadd_rn(c.x, __dmul_rn(r, t)));
}

// Integer part of a double y >= 0 (below 2^63) from its bits: y = m 2^e with
// the 53-bit significand m, so trunc(y) = m >> -e or m << e.  The same value
// as the conversion instruction, without the FP64 pipe (where GB300's
// double-to-integer conversions and roundings run at the FP64 rate).
__device__ __forceinline__ long long trunc_nonneg(double y) {
  const long long b = __double_as_longlong(y);
  const int e = (int)(b >> 52) - 1075;
  const long long m = (b & 0x000fffffffffffffLL) | 0x0010000000000000LL;
  if (e < -52) return 0;
  return e >= 0 ? (m << e) : (m >> -e);
}

// Sign tests and clamps of doubles on their bits (integer operations; the
// same results as the floating-point ones for numbers, zeros included)
__device__ __forceinline__ bool dpos(double x) { return __double_as_longlong(x) > 0; }  // x > 0
__device__ __forceinline__ bool dzero(double x) { return (__double_as_longlong(x) << 1) == 0; }
__device__ __forceinline__ double dmax0(double x) {                                    // max(0, x)
  return __double_as_longlong(x) < 0 ? 0.0 : x;
}
__device__ __forceinline__ double dclamp1(double x) {                                 // to [-1, 1]
  const long long b = __double_as_longlong(x);
  return (b & 0x7fffffffffffffffLL) > 0x3ff0000000000000LL
             ? __longlong_as_double((b & (long long)0x8000000000000000ULL) | 0x3ff0000000000000LL)
             : x;
}
// a < b for a, b >= 0 (doubles: on the bits; floats: the FP32 compare)
__device__ __forceinline__ bool lt_nn(double a, double b) {
  return __double_as_longlong(a) < __double_as_longlong(b);
}
__device__ __forceinline__ bool lt_nn(float a, float b) { return a < b; }
// |x| < t for t > 0
__device__ __forceinline__ bool dabs_lt(double x, double t) {
  return (__double_as_longlong(x) & 0x7fffffffffffffffLL) < __double_as_longlong(t);
}

// x (finite, >= 0) truncated to FP32 from its bits: a search hint, not a value
__device__ __forceinline__ float dtof_hint(double x) {
  const long long b = __double_as_longlong(x);
  const long long e = (b >> 52) - 1023 + 127;
  if (e <= 0) return 0.0f;
  if (e >= 255) return 3.0e38f;
  return __int_as_float((int)((e << 23) | ((b >> 29) & 0x7fffff)));
}

// floor(x) for x < 2^31 as an int, -1 for every negative x (callers clamp
// below at 0), by the sign bit and trunc_nonneg
__device__ __forceinline__ int floor_or_m1(double x) {
  return __double_as_longlong(x) < 0 ? -1 : (int)trunc_nonneg(x);
}

// uniforms from the top bits of a 64-bit word
__device__ __forceinline__ double u01d(unsigned long long w) {
  return u53_scaled(w >> 11, 53);                        // 53 bits; 0 maps to 0.0
}
__device__ __forceinline__ double eta01d(unsigned long long w) {
  return u53_scaled((w >> 11) + 1, 53);                  // in (0, 1]
}
__device__ __forceinline__ float u01f(unsigned long long w) {
  return (float)(unsigned)(w >> 40) * (1.0f / 16777216.0f);
}
__device__ __forceinline__ float eta01f(unsigned long long w) {
  return (float)((unsigned)(w >> 40) + 1u) * (1.0f / 16777216.0f);
}

// ------------------------------------------------------------------------
// memory-model helpers

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ long long ld_relaxed_s(const long long* p) {
  long long v;
  asm volatile("ld.relaxed.gpu.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_i(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

}  // namespace karl
