/*
 * karl.h - C ABI of the GB300 (sm_103a) KARL transport hot path.
 *
 * KARL follows beta-decay electrons and their secondary electrons and ions
 * through the tritium source along the magnetic-field axis (Sec. 2.1 main
 * cycle, Fig. 1).  Each step samples a free path from the local gas density
 * and the total cross section (Eqs. mean_free_path and distance_from_mfp),
 * picks a channel with probability sigma_i n_i / sum_j sigma_j n_j, performs
 * it (Sec. 3.3: elastic, ionization, excitation, clustering, recombination),
 * spawns products, and adds to the end-spectrum, density (Sec. 2.2, Eq.
 * target_field_density) and current (Sec. 2.3) tallies and to the
 * recombination target fields.  All of it runs in CUDA kernels on one GPU.
 *
 * Conventions for every entry point:
 *  - units are SI (m, m^-3, m^2, s, T) except energies in eV;
 *  - the caller owns every buffer it passes; create() copies what it needs;
 *  - no exception crosses the ABI: every error is a karl_status, and the
 *    context stays usable after KARL_EINVAL, KARL_ETIMEOUT, KARL_ECAPACITY and
 *    KARL_ECANCELLED;
 *  - a context is used by one host thread at a time;
 *  - pointers marked "host or device" are device pointers when the struct's
 *    on_device field is 1, host pointers otherwise.
 */
#ifndef KARL_H
#define KARL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct karl_ctx karl_ctx;

typedef enum karl_status {
  KARL_OK = 0,
  KARL_EINVAL = 1,      /* invalid argument or inconsistent tables */
  KARL_ENOMEM = 2,      /* device or pinned allocation failed */
  KARL_ECUDA = 3,       /* CUDA runtime error (the message has the detail) */
  KARL_ETIMEOUT = 4,    /* the transport kernel hit its time limit and stopped */
  KARL_EOVERFLOW = 5,   /* a 64-bit tally would overflow */
  KARL_ECAPACITY = 6,   /* particle queue too small even after regrowth */
  KARL_ECANCELLED = 7,  /* karl_cancel() was called during the run */
  KARL_EBUSY = 8,       /* server queue full */
  KARL_ENOTFOUND = 9    /* unknown request id */
} karl_status;

enum { KARL_N_SPECIES = 4, KARL_N_REASONS = 8, KARL_LEDGER_LEN = 64, KARL_MAX_CHANNELS = 16 };

/* tracked species (Sec. 3.8, Species: electron, T2+, T3+, T+) */
enum { KARL_ELECTRON = 0, KARL_T2P = 1, KARL_T3P = 2, KARL_TP = 3 };

/* interaction kinds (Sec. 3.3) */
enum {
  KARL_ELASTIC = 0,        /* energy conserved in the CM frame, isotropic CM angle */
  KARL_IONIZATION = 1,     /* E -> E - I - W, secondary electron W, ion species_out */
  KARL_EXCITATION = 2,     /* E -> E - loss, direction unchanged */
  KARL_CLUSTERING = 3,     /* ion -> species_out with a thermal target's energy */
  KARL_RECOMBINATION = 4,  /* impactor deleted; species_out = partner field */
  /* Sec. 3.3 Charge exchange: the ion (species_in not an electron) takes the
   * velocity of a target particle, drawn as for a moving elastic target (gas
   * drift plus Maxwell-Boltzmann, relative-speed weight); species kept,
   * species_out unused, the change of kinetic energy goes to the gas */
  KARL_CHARGE_EXCHANGE = 5,
  /* Sec. 3.3 Clustering, Eq. clustering_tertiary: three-body clustering,
   * rate per unit path sigma(E) n(z)^2 with the table holding k_ter / v(E)
   * (m^5), so the mean free path is v / (k_ter n^2); product as CLUSTERING */
  KARL_CLUSTERING3 = 6
};

/* termination reasons (Sec. 3.2 terminator and deletion logger) */
enum {
  KARL_R_EXIT0 = 0, KARL_R_EXIT1 = 1, KARL_R_CUTOFF = 2, KARL_R_CAP_COLL = 3,
  KARL_R_CAP_TIME = 4, KARL_R_RECOMB = 5, KARL_R_CLUSTER = 6, KARL_R_STALLED = 7
};

/* ledger slots (int64).  Energies in units of 2^-24 eV; per history and in
 * total  IN_PRIMARY + IN_THERMAL == sum(EXIT0 .. STALLED)  holds exactly, and
 * births[s] == sum_r deaths[s][r]. */
enum {
  KARL_L_E_IN_PRIMARY = 0, KARL_L_E_IN_THERMAL = 1, KARL_L_E_EXIT0 = 2, KARL_L_E_EXIT1 = 3,
  KARL_L_E_CUTOFF = 4, KARL_L_E_CAP = 5, KARL_L_E_RECOMB = 6, KARL_L_E_CLUSTER = 7,
  KARL_L_E_LOSS_IONIZ = 8, KARL_L_E_LOSS_EXCIT = 9, KARL_L_E_LOSS_RECOIL = 10,
  KARL_L_E_STALLED = 11,
  KARL_L_BIRTHS = 12,        /* [4] */
  KARL_L_DEATHS = 16,        /* [4][8] */
  KARL_L_N_COLLISIONS = 48, KARL_L_N_FLIGHTS = 49, KARL_L_N_SPAWN_E = 50, KARL_L_N_SPAWN_ION = 51,
  /* collisions and flights of every pass that wrote this ledger: both passes of
   * a two-pass karl_run or served request (whose other slots hold the last
   * pass), the sum over the cycles of karl_run_cycles, and the pass itself for
   * karl_run_pass, karl_run_cycle and karl_run_pass_static (added to out) */
  KARL_L_N_COLLISIONS_ALL = 52, KARL_L_N_FLIGHTS_ALL = 53
};

/* Geometry, gas and terminator settings (copied at create).
 * The source is a column [0, length_m] cut into n_zbins equal segments (the
 * density-field segmentation of Sec. 2.2); the gas density is constant in
 * each segment.  B is uniform along z, so the guiding-centre motion is
 * exact (Sec. 3.1, drift mover) and only z and the pitch cosine are tracked. */
typedef struct karl_geometry {
  double length_m;             /* > 0 */
  int32_t n_zbins;             /* 1 .. 1<<20 */
  const double* n_seg_m3;      /* host, [n_zbins], >= 0 */
  double area_m2;              /* face area A and segment volume A*dz, > 0 */
  double activity_bq;          /* a of Eq. simulated_time, > 0 */
  double e_cut_ev;             /* electrons below this energy are terminated */
  uint32_t max_collisions;     /* terminator cap on interactions per particle */
  double max_lifetime_s;       /* terminator cap on time alive (INFINITY = none) */
  double gas_temperature_k;    /* thermal target for ion products */
  int32_t n_tebins;            /* log-E bins of the time (density) tally, >= 1 */
  int32_t n_spec_bins;         /* end-spectrum bins (one overflow bin added) */
  double spec_bin_ev;          /* end-spectrum bin width, > 0 */
  double species_mass_ev[KARL_N_SPECIES];   /* rest energies */
  double target_mass_ev;       /* background gas molecule */
  double gas_drift_mps;        /* drift velocity of the gas along +z (moving targets) */
} karl_geometry;

/* Scattering-angle distributions of elastic channels (copied at create).
 * Sec. 3.3 (Elastic): the centre-of-mass polar angle chi is isotropic, drawn
 * from a tabulated distribution, or from a composition of the two that is
 * isotropic below a threshold energy.  A set s holds, for each of n_bins
 * impact-energy bins log-spaced over [e_min_ev[s], e_max_ev[s]] (bin
 * floor(n_bins ln(E/e_min)/ln(e_max/e_min)), clamped to the first and last),
 * the pdf of cos chi at n_mu points evenly spaced over [-1, 1]; between the
 * points the pdf is linear, and cos chi is drawn by inverting its cumulative
 * integral.  Below threshold_ev[s] the angle is isotropic.  The impact energy
 * is the lab energy for a target at rest and the relative kinetic energy of
 * the impactor for a moving target.
 * Errors (KARL_EINVAL at create): n_sets outside 1 .. KARL_MAX_CHANNELS,
 * n_bins < 1, n_mu < 2 or > 4096, a set index outside [-1, n_sets), a set on a
 * channel that is not elastic, e_min <= 0 or e_max <= e_min, a negative or
 * non-finite threshold or pdf value, or a bin whose pdf integrates to zero. */
typedef struct karl_angular {
  int32_t n_sets, n_bins, n_mu;
  const int32_t* set;          /* host, [n_channels]: -1 isotropic, else the set index */
  const double* e_min_ev;      /* host, [n_sets] */
  const double* e_max_ev;      /* host, [n_sets] */
  const double* threshold_ev;  /* host, [n_sets] */
  const double* pdf;           /* host, [n_sets][n_bins][n_mu], >= 0 (need not be normalised) */
} karl_angular;

/* Cross-section tables (copied at create).  sigma of channel k at energy E is
 * linear in ln E between the log-spaced nodes e_min * (e_max/e_min)^(i/(n-1)),
 * clamped outside, and zero for E <= loss_ev[k] (Sec. 3.3: the cross section
 * is a one-dimensional functional of the energy). */
typedef struct karl_xs {
  int32_t n_energy;            /* >= 2 */
  double e_min_ev, e_max_ev;   /* 0 < e_min < e_max */
  /* 0 .. KARL_MAX_CHANNELS, selection order; per impactor species at most 10
   * channels, of which at most 2 have a rate that follows a field other than
   * n(z) (recombination, three-body clustering) */
  int32_t n_channels;
  const int32_t* kind;         /* host, [n_channels] */
  const int32_t* species_in;   /* host, impactor species */
  const int32_t* species_out;  /* host, see the kinds above; -1 = none */
  const double* loss_ev;       /* host, threshold / energy loss (>= 0) */
  const double* sigma_m2;      /* host, [n_channels][n_energy], >= 0 */
  double ioniz_eps_ev;         /* eps of the secondary-energy pdf 1/(1+(W/eps)^2) */
  /* host, [n_channels] or NULL (all 0): 0 = target at rest; 1 = moving target
   * (Sec. 3.3 Elastic: the gas drift plus a Maxwell-Boltzmann velocity at the
   * gas temperature, drawn with the relative-speed weight of the collision
   * rate; the impactor turned in the centre-of-mass frame.  Sec. 3.3
   * Ionization: the target drawn the same way and redrawn while the impact
   * energy relative to it is not above the ionization energy; the energy
   * shared and the angles drawn in the target's frame; the ion leaves with
   * the target velocity; the lab energy the gas gives or takes is booked as
   * recoil).  1 is allowed for elastic and ionization channels. */
  const int32_t* target;
  /* host or NULL (every elastic channel isotropic in the centre-of-mass frame) */
  const karl_angular* angular;
} karl_xs;

/* Primary particles (one beta electron and, with ions, one T2+ per decay,
 * Sec. 3.5).  Primary id = pid_offset + index keys the random streams, so a
 * run split into id ranges sums to the same tallies bit for bit. */
typedef struct karl_primaries {
  int64_t n;                   /* >= 0 */
  const double* z_m;           /* host or device, [n], 0 <= z <= length */
  const double* e_ev;          /* host or device, [n], > 0 */
  const double* mu;            /* host or device, [n], -1 <= mu <= 1 */
  const uint8_t* species;      /* host or device, [n] */
  int64_t n_decays;            /* decays of the whole run: t_sim = n_decays / activity */
  int64_t pid_offset;
  int32_t on_device;
} karl_primaries;

/* Output tallies (caller-owned, zeroed by the run).  Layouts are row-major. */
typedef struct karl_tallies {
  uint64_t* spectrum;          /* [2][4][n_spec_bins+1] particles leaving at z=0 / z=L */
  uint64_t* time_fx;           /* [4][n_zbins+2][n_tebins] time in segment, LSB 2^-50 s;
                                  rows 0 and n_zbins+1 are the under/overflow bins */
  uint64_t* cross_pos;         /* [4][n_zbins+1] face crossings towards +z */
  uint64_t* cross_neg;         /* [4][n_zbins+1] face crossings towards -z */
  uint64_t* recomb;            /* [4][n_zbins] deletions logged in each species' field */
  int64_t* ledger;             /* [KARL_LEDGER_LEN] */
  uint64_t* chan_count;        /* [n_channels] collisions per channel */
  uint64_t* per_primary;       /* [n] collisions in each primary's tree, or NULL */
  double* density;             /* [4][n_zbins] Eq. target_field_density, or NULL */
  double* current;             /* [4][n_zbins+1] (N+ - N-)/(A t_sim), or NULL */
  double* field;               /* [4][n_zbins][n_tebins] pass-1 densities, or NULL */
  int32_t on_device;
} karl_tallies;

enum { KARL_FP64 = 0, KARL_FP32 = 1 };

typedef struct karl_run_opts {
  uint64_t seed;
  int32_t n_passes;            /* 1, or 2 when recombination channels exist */
  int32_t precision;           /* KARL_FP64 (plain) or KARL_FP32 (precision form) */
  int32_t block_size;          /* threads per block, a multiple of 32 up to 512; 0 = default */
  int32_t blocks_per_sm;       /* 0 = occupancy maximum */
  double timeout_s;            /* kernel time limit; <= 0 = 600 s */
  void* stream;                /* cudaStream_t, NULL = the context's own stream */
} karl_run_opts;

/* Validate and copy geometry and tables to the current CUDA device.
 * Errors: KARL_EINVAL (any field out of range, NULL table), KARL_ENOMEM,
 * KARL_ECUDA.  *out is NULL on error. */
karl_status karl_create(const karl_geometry* geom, const karl_xs* xs, karl_ctx** out);

/* Whole run: pass 1 (no recombination) and, if n_passes == 2, pass 2 with
 * the target fields frozen from pass 1 (Eq. target_field_density, Sec. 3.6
 * additive fields).  Tallies of the last pass are returned, normalised
 * density/current from them, and the pass-1 densities as `field`.
 * Blocks until done (the work is ordered on opts->stream).
 * Errors: KARL_EINVAL, KARL_ENOMEM, KARL_ECUDA, KARL_ETIMEOUT, KARL_ECAPACITY,
 * KARL_ECANCELLED; on error the tallies are unspecified. */
karl_status karl_run(karl_ctx* ctx, const karl_primaries* prim, const karl_run_opts* opts,
                     karl_tallies* out);

/* One pass over a primary-id range, raw integer tallies only, ADDED to out
 * (density/current/field untouched).  pass = 2 builds the target fields from
 * field_time_in (host, [4][n_zbins+2][n_tebins], the pass-1 time tallies
 * summed over every shard) and prim->n_decays.  This is the host-side
 * exchange step of a run split over ranks (Sec. 3.6: additive sync). */
karl_status karl_run_pass(karl_ctx* ctx, const karl_primaries* prim, const karl_run_opts* opts,
                          int32_t pass, const uint64_t* field_time_in, karl_tallies* out);

/* The paper's continuous field update (Sec. 3.6): the primaries run in
 * n_cycles consecutive cycles, cycle c over indices [c n / C, (c+1) n / C),
 * each with the target fields of every cycle before it -- Eq.
 * target_field_density over their summed time tallies, with the -N/V term of
 * the recombination deletions logged in the partner's field (a bin's density
 * takes the segment's deletions in proportion to its time there, and counts
 * as zero below zero), t_sim (Eq. simulated_time) from their share of
 * prim->n_decays -- and the first cycle with fields of zero.  All cycles draw
 * from the pass-2 random streams, so without recombination channels the
 * result does not depend on n_cycles.  Returns in out the raw tallies summed
 * over the cycles, the density and current of the whole run, and as `field`
 * the per-bin densities (deletions included) a next cycle would use.
 * opts->n_passes is ignored.  Errors: those of karl_run, KARL_EINVAL for
 * n_cycles < 1. */
karl_status karl_run_cycles(karl_ctx* ctx, const karl_primaries* prim, const karl_run_opts* opts,
                            int32_t n_cycles, karl_tallies* out);

/* One cycle of the continuous update over a primary-id range, raw tallies
 * ADDED to out (the building block of karl_run_cycles for runs split over
 * ranks): recombination on, with the fields of field_time_in (host,
 * [4][n_zbins+2][n_tebins]) and field_recomb_in (host, [4][n_zbins], or NULL
 * for no deletions) summed over the earlier cycles of every rank, t_sim =
 * field_decays / activity; field_time_in NULL: fields of zero (the first
 * cycle).  Errors: those of karl_run_pass, KARL_EINVAL for field_decays <= 0
 * with fields given. */
karl_status karl_run_cycle(karl_ctx* ctx, const karl_primaries* prim, const karl_run_opts* opts,
                           const uint64_t* field_time_in, const uint64_t* field_recomb_in,
                           double field_decays, karl_tallies* out);

/* ---------------------------------------------------------------------------
 * One pass that allocates nothing.  The paper has no counterpart: this is a
 * deployment form of karl_run_pass, with the same kernel and results.
 *
 * Who needs it: callers that may not allocate device memory while they run --
 * a host framework whose caching allocator or fixed budget has reserved the
 * GPU's memory up front, or a request path that keeps cudaMalloc/cudaFree (and
 * the device-wide synchronisation they can cause) out.  karl_run_pass grows
 * work buffers on demand (tally staging, the particle ring, regrown on
 * overflow); this call places all of its scratch in one static device array
 * of KARL_STATIC_SCRATCH_BYTES per device that the library image carries, and
 * reads and writes only caller-owned device memory.  It calls no allocating
 * routine (no cudaMalloc, cudaFree, or library routine that allocates).
 *
 * Arguments as karl_run_pass, except:
 *  - prim->on_device and out->on_device must be 1 (device pointers only), and
 *    for pass 2 field_time_in is a DEVICE array [4][n_zbins+2][n_tebins];
 *  - the pass's raw integer tallies OVERWRITE out's buffers (the call zeroes
 *    them first) where karl_run_pass adds to them; per_primary may be NULL;
 *    density, current and field are not touched.
 * Scratch: control block, time and crossing difference arrays, pass-2 field
 * tables, and a particle ring of 64-byte cells that gets the rest.  The fixed
 * part is about 2 * 4 * (n_zbins + 2) * n_tebins * 8 bytes (time) +
 * 2 * 4 * (n_zbins + 2) * 8 bytes (crossings) + for pass 2
 * 2 * n_channels * (n_zbins + 1) * 8 bytes (field tables); the ring is the
 * largest power of two of cells with fixed + 64 * cells <= 64 MiB, from 2^16
 * up to 2^19 cells (2^19 for config-sized geometries, 1000 segments and 64
 * energy bins).  karl_run_pass starts at 2^22 cells and grows on overflow, so
 * a workload that succeeds there can fail here: a geometry whose fixed part
 * does not fit beside the smallest ring (4 MiB) is rejected with
 * KARL_ECAPACITY before any launch, and so is a run whose particles overflow
 * the ring, which cannot grow here.
 * Pointers: every primary array, tally buffer and field_time_in must be device
 * (or managed) memory of the context's device; anything else is rejected with
 * KARL_EINVAL before any launch (checked with cudaPointerGetAttributes).
 * Set-up: the first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture on the device.
 * Concurrency: one scratch array per device is shared by every context of the
 * process.  Calls on the same device that overlap in time (two threads, or two
 * streams without an order between them) race on it and corrupt each other's
 * results: serialise them.
 * Blocks until the pass is done.  Errors: those of karl_run_pass, plus
 * KARL_EINVAL for host buffers and KARL_ECAPACITY as above; karl_cancel
 * applies.  On error the tallies are unspecified. */
#define KARL_STATIC_SCRATCH_BYTES (64u << 20)
karl_status karl_run_pass_static(karl_ctx* ctx, const karl_primaries* prim,
                                 const karl_run_opts* opts, int32_t pass,
                                 const uint64_t* field_time_in, karl_tallies* out);

/* ---- Full-orbit transport in a beam tube (Sec. 3.1 Boris mover) ----
 *
 * Each particle carries its position (x, y, z) and proper velocity
 * u = gamma v.  A step is one relativistic Boris push (Sec. 3.1: half an
 * electric kick, the magnetic rotation, half a kick; the paper's equations
 * with u = gamma v and gamma of the half-kicked velocity) with the species'
 * time step in the uniform field b_t along +z and the electric field
 * E = (e_r_vm2 x, e_r_vm2 y, e_z_vm[segment of z]).  The initial velocity is
 * the half-step velocity.  A flight draws eta once and ends where the optical
 * depth summed over its steps (the total rate of the step midpoint's segment
 * times the step's path length; cross sections at the flight's starting
 * energy without electric field, at each step's energy with one) reaches
 * -ln eta, at z = 0 or L, where the path meets the wall r = tube_radius_m,
 * or at the lifetime cap; that last step is shortened to the fraction of its
 * displacement where it happens (on a tie: wall, z end, lifetime, collision).
 * Collisions use the context's tables and the kinematics of Sec. 3.3 with
 * directions turned in three dimensions (frame: the unit vector towards +z
 * normal to the old direction, so the pitch update equals the guiding-centre
 * one).  Channel kinds: elastic and ionization with the target at rest,
 * excitation, clustering, three-body clustering; recombination, charge
 * exchange and moving targets are refused (KARL_EINVAL).  Energies are FP64
 * and not quantised (an electric field changes them continuously).
 * Tallies are raw and ADDED to out's buffers (zero them first):
 *   time_z [4][n_zbins], time_r [4][n_rbins]: time per z segment and per
 *     radial bin (width R / n_rbins), u64 in units of 2^-50 s; the time of a
 *     step goes to the cell of its midpoint, each run of steps in one cell
 *     rounded once;
 *   cross_pos / cross_neg [4][n_zbins+1]: crossings of z faces (the end faces
 *     count the exits);
 *   rcross_out / rcross_in [4][n_rbins+1]: crossings of the cylinders
 *     r = k R / n_rbins between the radial bins of a step's ends (k = n_rbins:
 *     the wall, outward only);
 *   wall [4][n_zbins]: particles ended on the wall, by z segment (Sec. 5's
 *     tube current);
 *   spectrum [2][4][n_spec_bins+1]: kinetic energies at z = 0 and z = L in
 *     bins of spec_bin_ev, the last bin collecting the overflow;
 *   ledger [KARL_ORBIT_LEDGER] int64, energy [KARL_ORBIT_ENERGY] double:
 *     slots below; chan_count [n_channels];
 *   per_primary [n] (may be NULL): collisions in each primary's tree;
 *   end_state [n][8] (may be NULL): x y z E ux uy uz t of each primary when
 *     it ended (its clustering, for an ion that clusters).
 * Every buffer is host memory.  opts: precision must be KARL_FP64, n_passes
 * is ignored; block_size 0 = 256 (at most 256); timeout_s limits each of the
 * kernel launches (one per product generation).  Errors: KARL_EINVAL (NULL
 * or inconsistent arguments, a primary outside the tube or the column, a
 * refused channel kind); KARL_ECAPACITY when one generation's products
 * exceed max(2^20, 8 n_in) slots or more than 4096 generations are needed
 * (tallies unspecified); KARL_ETIMEOUT; KARL_ECANCELLED (karl_cancel). */
enum {
  KARL_OB_BIRTHS = 0,           /* [4] */
  KARL_OB_DEATHS = 4,           /* [4][8] by reason: exit z=0, exit z=L, wall, cutoff,
                                   collision cap, lifetime cap, clustering, stalled */
  KARL_OB_N_COLLISIONS = 36, KARL_OB_N_FLIGHTS = 37, KARL_OB_N_STEPS = 38,
  KARL_OB_N_SPAWN_E = 39, KARL_OB_N_SPAWN_ION = 40,
  KARL_ORBIT_LEDGER = 48
};
enum {
  KARL_OE_IN_PRIMARY = 0, KARL_OE_IN_THERMAL = 1, KARL_OE_EXIT0 = 2, KARL_OE_EXIT1 = 3,
  KARL_OE_WALL = 4, KARL_OE_CUTOFF = 5, KARL_OE_CAP = 6, KARL_OE_CLUSTER = 7,
  KARL_OE_LOSS_IONIZ = 8, KARL_OE_LOSS_EXCIT = 9, KARL_OE_RECOIL = 10, KARL_OE_STALLED = 11,
  KARL_OE_FIELD_WORK = 12,      /* kinetic energy gained from the electric field */
  KARL_ORBIT_ENERGY = 16
};
typedef struct karl_orbit {
  double b_t;                   /* magnetic field along +z (T) */
  double tube_radius_m;         /* wall radius R > 0 */
  int32_t n_rbins;              /* radial bins, 1 .. 2^20 */
  int32_t pad;
  const double* e_z_vm;         /* [n_zbins] axial field per segment (V/m), NULL: none */
  double e_r_vm2;               /* radial field E_r = e_r_vm2 r (V/m^2) */
  double dt_s[4];               /* Boris time step per species, > 0 */
  uint64_t max_steps;           /* steps of one flight before the particle counts as
                                   stalled; 0 = 2^40 */
} karl_orbit;
typedef struct karl_orbit_primaries {
  int64_t n;
  const double* x_m;
  const double* y_m;
  const double* z_m;            /* inside the tube: x^2 + y^2 < R^2, 0 <= z <= L */
  const double* e_ev;
  const double* mu;             /* cosine of the angle to +z */
  const double* phi;            /* azimuth of the transverse velocity (rad) */
  const uint8_t* species;
  int64_t pid_offset;           /* primary id of element 0 (random streams) */
} karl_orbit_primaries;
typedef struct karl_orbit_tallies {
  uint64_t* spectrum;
  uint64_t* time_z;
  uint64_t* time_r;
  uint64_t* cross_pos;
  uint64_t* cross_neg;
  uint64_t* rcross_out;
  uint64_t* rcross_in;
  uint64_t* wall;
  int64_t* ledger;
  double* energy;
  uint64_t* chan_count;
  uint64_t* per_primary;
  double* end_state;
} karl_orbit_tallies;
karl_status karl_run_orbit(karl_ctx* ctx, const karl_orbit* orbit,
                           const karl_orbit_primaries* prim, const karl_run_opts* opts,
                           karl_orbit_tallies* out);

/* Request that a running karl_run on this context stop (thread-safe).  The
 * kernel polls the flag; the run returns KARL_ECANCELLED. */
void karl_cancel(karl_ctx* ctx);

/* Sizes of the tally arrays (elements) for buffer allocation. */
typedef struct karl_layout {
  int64_t spectrum, time_fx, cross, recomb, ledger, chan_count, density, current, field;
} karl_layout;
karl_status karl_tally_layout(const karl_ctx* ctx, karl_layout* out);

/* Statistics of the last run on this context. */
typedef struct karl_run_stats {
  double kernel_ms[2];         /* transport kernel time per pass (CUDA events) */
  int64_t collisions[2];
  int64_t flights[2];
  int64_t particles[2];        /* particles processed (primaries + products) */
  double lane_occupancy[2];    /* mean fraction of lanes holding a particle */
  int32_t grid_blocks, block_size;
  int32_t queue_capacity;
  int64_t kernel_launches;
  /* per pass: device time from the claim of the last primary to the end of
   * the launch (the pass tail, when lanes run out of work), and the products
   * that went through the shared device ring rather than a warp's queue */
  double tail_ms[2];
  int64_t spilled[2];
  /* per pass: share of warp iterations in which the warp held no particle */
  double idle_warp_frac[2];
} karl_run_stats;
karl_status karl_last_stats(const karl_ctx* ctx, karl_run_stats* out);

/* Free everything the context owns.  NULL is ignored. */
void karl_destroy(karl_ctx* ctx);

/* Static description of a status code. */
const char* karl_status_string(karl_status s);

/* Detail of the last error on this context (empty if none). */
const char* karl_last_error(const karl_ctx* ctx);


/* ------------------------------------------------------------------------
 * Many requests in one persistent launch (batched and served forms).
 *
 * A server holds one physics model (the cross-section tables and species of
 * karl_xs) and runs requests, each with its own geometry, gas profile,
 * primaries and seed, as independent source configurations of the same
 * transport step (Sec. 2.1).  Requests are admitted while their device
 * footprint fits the server's HBM budget and a slot is free; admitted
 * requests join the running kernel (continuous batching) and move through
 * pass 1, target fields and pass 2 on the device.  Each request's result is
 * the same alone or in any mix: its random streams are keyed by its seed and
 * primary ids only.
 *
 * A batch is a server whose requests are all submitted before
 * karl_server_run_all(), which publishes them, runs them in one persistent
 * launch and collects every result.  The server API is not thread-safe:
 * serialise calls on one server.
 *
 * A launch holds every SM of the device from the first admitted request
 * until karl_server_run_all() or karl_server_destroy() closes it.  Meanwhile
 * other kernels on the device (a karl_run, a memset, another library's work)
 * wait for it, and so do calls that synchronise the whole device
 * (cudaDeviceSynchronize, cudaFree).  Contexts take their device memory from
 * a stream-ordered pool, so creating and destroying them does not wait.
 */
typedef struct karl_server karl_server;

typedef struct karl_server_opts {
  int32_t precision;           /* KARL_FP64 or KARL_FP32 */
  int32_t max_slots;           /* requests on the device at once, 1 .. 1024 (0 = 256) */
  int64_t hbm_budget_bytes;    /* device arena for request state (0 = 16 GiB) */
  double timeout_s;            /* limit on one persistent launch (<= 0: 3600 s) */
  int32_t block_size;          /* 0 = 256 */
  int32_t blocks_per_sm;       /* 0 = occupancy maximum */
} karl_server_opts;

/* Create a server for the model in xs (tables copied).  Species masses,
 * target mass, and the energy grid of the time tally come from each request's
 * geometry.  Errors: KARL_EINVAL, KARL_ENOMEM, KARL_ECUDA. */
karl_status karl_server_create(const karl_xs* xs, const karl_server_opts* opts,
                               karl_server** out);

/* Queue one request (geometry and primaries copied; host pointers only).
 * Its results will be written into out: host buffers (on_device = 0) sized
 * as karl_tally_layout gives for this geometry, owned by the caller and kept
 * valid until karl_server_poll reports the request done; per_primary is not
 * used.  n_passes as in karl_run_opts.  The request is admitted at once if a
 * slot and arena space are free, else as earlier requests finish.
 * Errors: KARL_EINVAL (bad geometry, primaries, buffers, more than 2^31 - 1
 * primaries, or a footprint larger than the whole budget), KARL_ENOMEM. */
karl_status karl_server_submit(karl_server* srv, const karl_geometry* geom,
                               const karl_primaries* prim, uint64_t seed, int32_t n_passes,
                               karl_tallies* out, uint64_t* req_id);

/* Non-blocking: collects every finished request (copies its tallies into the
 * caller's buffers, releases its device state), admits waiting requests, and
 * sets *done = 1 if req_id has finished.  A finished id stays known until
 * polled once with done = 1.  Errors: KARL_ENOTFOUND (unknown id),
 * KARL_ETIMEOUT / KARL_ECANCELLED (the launch stopped before it finished),
 * KARL_ECUDA. */
karl_status karl_server_poll(karl_server* srv, uint64_t req_id, int* done);

/* Size of each output array of a request with this geometry (elements). */
karl_status karl_server_layout(const karl_server* srv, const karl_geometry* geom,
                               karl_layout* out);

/* Batch: admit, run and finish every submitted request in as few persistent
 * launches as the HBM budget allows (one when everything fits), blocking
 * until the last result is in the caller's buffers. */
karl_status karl_server_run_all(karl_server* srv);

typedef struct karl_server_stats {
  int64_t submitted, admitted, completed, collected, waiting;
  int64_t collisions;          /* collisions of every pass, summed over collected requests */
  int64_t kernel_launches;
  int64_t arena_bytes_in_use, arena_bytes_peak;
  double lane_occupancy;       /* of the last finished launch */
  double kernel_ms;            /* device time of the finished launches (CUDA events) */
} karl_server_stats;
karl_status karl_server_get_stats(const karl_server* srv, karl_server_stats* out);

/* Stop the running launch after the published requests finish, free all
 * device state.  NULL is ignored. */
void karl_server_destroy(karl_server* srv);

/* Detail of the last server error (empty if none). */
const char* karl_server_last_error(const karl_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* KARL_H */
