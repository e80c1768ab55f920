/*
 * karl_oracle.h - plain FP64 CPU oracle of the KARL transport step.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the correctness reference for the
 * CUDA path.  Only the tests, __graft_entry__.smoke() and bench.py's CPU
 * baseline may load it; the product path never calls it.
 *
 * It follows the paper event by event (Sec. 2.1 main cycle and Fig. 1, the
 * free-path law Eqs. mean_free_path / distance_from_mfp, the segment-stop
 * mover rule of Sec. 3.1, the interactions of Sec. 3.3, the density-field and
 * current estimators of Secs. 2.2-2.3 and Eq. target_field_density) in FP64.
 * It shares no code with the GPU path.
 *
 * Pins (tests/test_oracle_*.py) fix every step against closed forms,
 * quadrature, library routines and exact invariants.  The whole-run tallies
 * of the full configurations (orc_run on configs 1 and 2) have no closed
 * form: parity unpinned beyond their pinned parts and the invariants (exact
 * ledgers, spectrum and crossing counts against deaths, shard additivity).
 */
#ifndef KARL_ORACLE_H
#define KARL_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_N_SPECIES = 4, ORC_N_REASONS = 8, ORC_LEDGER_LEN = 64 };

/* ledger layout (int64): energies in units of 2^-24 eV, then counters */
enum {
  ORC_E_IN_PRIMARY = 0, ORC_E_IN_THERMAL = 1, ORC_E_EXIT0 = 2, ORC_E_EXIT1 = 3,
  ORC_E_CUTOFF = 4, ORC_E_CAP = 5, ORC_E_RECOMB = 6, ORC_E_CLUSTER = 7,
  ORC_E_LOSS_IONIZ = 8, ORC_E_LOSS_EXCIT = 9, ORC_E_LOSS_RECOIL = 10, ORC_E_STALLED = 11,
  ORC_BIRTHS = 12,              /* [4] */
  ORC_DEATHS = 16,              /* [4][8] */
  ORC_N_COLLISIONS = 48, ORC_N_FLIGHTS = 49, ORC_N_SPAWN_E = 50, ORC_N_SPAWN_ION = 51,
  /* collisions and flights of every pass of the run (orc_run: both passes;
   * one pass: equal to ORC_N_COLLISIONS / ORC_N_FLIGHTS) */
  ORC_N_COLLISIONS_ALL = 52, ORC_N_FLIGHTS_ALL = 53
};

typedef struct {
  double length_m;
  int32_t n_zbins;
  const double* n_seg_m3;      /* [n_zbins] */
  double area_m2;
  double activity_bq;
  double e_cut_ev;
  uint32_t max_collisions;
  double max_lifetime_s;       /* +inf: no cap */
  double gas_temperature_k;
  int32_t n_tebins;
  int32_t n_spec_bins;
  double spec_bin_ev;
  double species_mass_ev[ORC_N_SPECIES];
  double target_mass_ev;
  int32_t n_energy;
  double e_min_ev, e_max_ev;
  int32_t n_channels;
  /* 0 elastic 1 ionization 2 excitation 3 clustering 4 recombination
     5 charge exchange 6 three-body clustering (rate sigma_k(E) n^2) */
  const int32_t* kind;
  const int32_t* species_in;
  const int32_t* species_out;
  const double* loss_ev;
  const double* sigma_m2;      /* [n_channels][n_energy] */
  double ioniz_eps_ev;
  /* per channel: 0 target at rest, 1 moving target (gas drift along +z plus a
     Maxwell-Boltzmann draw at the gas temperature; elastic and ionization
     channels); NULL: every target at rest */
  const int32_t* target;
  double gas_drift_mps;        /* drift velocity of the gas along +z */
  /* scattering-angle distributions of elastic channels (Sec. 3.3 Elastic):
     ang_set[k] = -1 (or ang_set NULL): isotropic in the centre-of-mass frame;
     otherwise the set used by channel k.  A set is a pdf of cos(chi) on
     ang_n_mu points evenly spaced over [-1, 1] (piecewise linear between
     them) for each of ang_n_bins log-spaced impact-energy bins over
     [ang_e_min_ev[s], ang_e_max_ev[s]]; below ang_threshold_ev[s] scattering
     is isotropic. */
  const int32_t* ang_set;
  int32_t ang_n_sets, ang_n_bins, ang_n_mu;
  const double* ang_e_min_ev;
  const double* ang_e_max_ev;
  const double* ang_threshold_ev;
  const double* ang_pdf;       /* [sets][bins][n_mu] */
} orc_problem;

typedef struct {
  int64_t n;
  const double* z_m;
  const double* e_ev;
  const double* mu;
  const uint8_t* species;
  int64_t n_decays;            /* decays of the whole run, for t_sim = N/a */
  int64_t pid_offset;          /* primary id of element 0 */
} orc_primaries;

typedef struct {
  uint64_t* spectrum;          /* [2][4][n_spec_bins+1] */
  uint64_t* time_fx;           /* [4][n_zbins+2][n_tebins], LSB 2^-50 s */
  uint64_t* cross_pos;         /* [4][n_zbins+1] */
  uint64_t* cross_neg;         /* [4][n_zbins+1] */
  uint64_t* recomb;            /* [4][n_zbins] */
  int64_t* ledger;             /* [ORC_LEDGER_LEN] */
  uint64_t* chan_count;        /* [n_channels] */
  uint64_t* per_primary;       /* [n] collisions in each primary's tree, may be NULL */
  double* density;             /* [4][n_zbins], may be NULL */
  double* current;             /* [4][n_zbins+1], may be NULL */
  double* field;               /* [4][n_zbins][n_tebins] pass-1 densities, may be NULL */
} orc_tallies;

/* mode 0: free flight by optical depth (one draw per flight);
 * mode 1: paper-literal segment stop and redraw (Sec. 3.1). */
int orc_run(const orc_problem* p, const orc_primaries* pr, uint64_t seed, int n_passes,
            int mode, int n_threads, orc_tallies* out);

/* One pass only.  pass = 1: no recombination.  pass = 2: recombination with
 * the target fields built from field_time_in (raw pass-1 time tallies of the
 * whole run, [4][n_zbins+2][n_tebins]).  Output tallies are raw and
 * accumulated (+=) into out; density/current/field are not written. */
int orc_run_pass(const orc_problem* p, const orc_primaries* pr, uint64_t seed, int pass,
                 const uint64_t* field_time_in, int mode, int n_threads, orc_tallies* out);

/* Test hooks. */
void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);
double orc_sigma(const orc_problem* p, int channel, double e_ev);
/* One collision of channel `channel` for a particle (species, e_ev, mu) with
 * the four uniforms u[0..3] as raw 64-bit words.  Returns the number of
 * products written to out_* (the incident particle first, if it survives). */
int orc_collide(const orc_problem* p, int channel, int species, double e_ev, double mu,
                const uint64_t words[4], double* out_e, double* out_mu, int* out_species);

/* Elastic collision with a moving target (the kinematics of a channel with
 * target == 1), for single-collision checks: the impactor (mass m1_ev, energy
 * e_ev, pitch cosine mu) meets a target whose velocity is drawn from Philox
 * blocks with counter (ctr[0], ctr[1], ctr[2], k) and key key[0..1]; w[2],
 * w[3] give the centre-of-mass angles.  Writes the impactor's energy and pitch
 * cosine after the collision, and (if not NULL) the velocities in units of c:
 * v[0..2] impactor before, v[3..5] target before, v[6..8] impactor after,
 * v[9..11] target after. */
void orc_elastic_moving_target(const orc_problem* p, double m1_ev, double e_ev, double mu,
                               const uint64_t w[4], const uint64_t ctr[3], const uint64_t key[2],
                               double* out_e, double* out_mu, double* v);

/* One cycle of the continuous field update (Sec. 3.6, Eq. target_field_density):
 * a pass with recombination whose target fields come from field_time_in
 * ([4][n_zbins+2][n_tebins]) and the deletions field_recomb_in ([4][n_zbins],
 * may be NULL) summed over the cycles before, with t_sim = field_decays /
 * activity; field_time_in NULL: every field zero.  Raw tallies are ADDED to
 * out.  Returns 0 on success. */
int orc_run_cycle(const orc_problem* p, const orc_primaries* pr, uint64_t seed,
                  const uint64_t* field_time_in, const uint64_t* field_recomb_in,
                  double field_decays, int mode, int n_threads, orc_tallies* out);

/* One ionization with a moving target (Sec. 3.3 Ionization) of channel
 * `channel`, impactor of rest energy m1_ev, kinetic energy e_ev and pitch
 * cosine mu, ion of rest energy m_ion_ev: w[2], w[3] share the energy and set
 * the azimuth; target velocities come from the blocks (ctr[0], ctr[1], ctr[2],
 * k) under key (redraw r: k from 128 r).  out: impactor energy and pitch
 * cosine, ejected electron energy and pitch cosine, ion energy and pitch
 * cosine, impact energy E_i (all eV). */
void orc_ionization_moving_target(const orc_problem* p, int channel, double m1_ev, double e_ev,
                                  double mu, double m_ion_ev, const uint64_t w[4],
                                  const uint64_t ctr[3], const uint64_t key[2], double out[7]);

/* One charge exchange (Sec. 3.3 Charge exchange) of an impactor of rest
 * energy m1_ev, kinetic energy e_ev and pitch cosine mu; the target velocity
 * is drawn from the blocks (ctr[0], ctr[1], ctr[2], k) under key.  Writes the
 * impactor's new energy and pitch cosine and, if v2 is not NULL, the target
 * velocity it took (units of c). */
void orc_charge_exchange(const orc_problem* p, double m1_ev, double e_ev, double mu,
                         const uint64_t ctr[3], const uint64_t key[2], double* out_e,
                         double* out_mu, double* v2);

/* cos(chi) of an elastic collision of channel `channel` at impact energy
 * e_ev for the uniform number u in [0, 1) (isotropic: 2u - 1). */
double orc_sample_angle(const orc_problem* p, int channel, double e_ev, double u);


/* ---- orbit mode: the Boris mover (Sec. 3.1) in a tube of radius R ----
 *
 * Full-orbit transport: position (x, y, z) and proper velocity u = gamma v are
 * advanced by the relativistic Boris push with the species' time step in a
 * uniform magnetic field b_t along +z and the electric field
 * E = (e_r_vm2 x, e_r_vm2 y, e_z_vm[segment of z]).  Flights end where the
 * optical depth accumulated over the steps reaches -ln(eta), at z = 0 or L,
 * on the tube wall r = R, or at the lifetime cap; the collision kinematics
 * are those of the guiding-centre path with the direction turned in three
 * dimensions.  Channels: elastic and ionization with the target at rest,
 * excitation, clustering and three-body clustering.  Energies are FP64 (no
 * quantisation: the electric field changes them continuously). */
enum {
  ORC_OB_BIRTHS = 0,            /* [4] */
  ORC_OB_DEATHS = 4,            /* [4][8], reasons below */
  ORC_OB_N_COLLISIONS = 36, ORC_OB_N_FLIGHTS = 37, ORC_OB_N_STEPS = 38,
  ORC_OB_N_SPAWN_E = 39, ORC_OB_N_SPAWN_ION = 40,
  ORC_OB_LEDGER_LEN = 48
};
enum { ORC_OR_EXIT0 = 0, ORC_OR_EXIT1 = 1, ORC_OR_WALL = 2, ORC_OR_CUTOFF = 3,
       ORC_OR_CAP_COLL = 4, ORC_OR_CAP_TIME = 5, ORC_OR_CLUSTER = 6, ORC_OR_STALLED = 7 };
/* energy ledger (eV, FP64) */
enum {
  ORC_OE_IN_PRIMARY = 0, ORC_OE_IN_THERMAL = 1, ORC_OE_EXIT0 = 2, ORC_OE_EXIT1 = 3,
  ORC_OE_WALL = 4, ORC_OE_CUTOFF = 5, ORC_OE_CAP = 6, ORC_OE_CLUSTER = 7,
  ORC_OE_LOSS_IONIZ = 8, ORC_OE_LOSS_EXCIT = 9, ORC_OE_RECOIL = 10, ORC_OE_STALLED = 11,
  ORC_OE_FIELD_WORK = 12,       /* kinetic energy gained from the electric field in flights */
  ORC_OE_LEN = 16
};

typedef struct {
  double b_t;                   /* uniform magnetic field along +z (T) */
  double tube_radius_m;         /* wall radius R; particles reaching it end there */
  int32_t n_rbins;              /* radial bins of width R / n_rbins */
  const double* e_z_vm;         /* [n_zbins] axial electric field per segment (V/m), NULL: 0 */
  double e_r_vm2;               /* radial electric field E_r = e_r_vm2 * r (V/m^2) */
  double dt_s[ORC_N_SPECIES];   /* Boris time step per species (s) */
  uint64_t max_steps;           /* steps per flight before a particle counts as stalled; 0: 2^40 */
} orc_orbit;

typedef struct {
  int64_t n;
  const double* x_m;
  const double* y_m;
  const double* z_m;
  const double* e_ev;
  const double* mu;             /* cosine of the angle to +z */
  const double* phi;            /* azimuth of the transverse velocity (rad) */
  const uint8_t* species;
  int64_t pid_offset;
} orc_orbit_primaries;

typedef struct {
  uint64_t* spectrum;           /* [2][4][n_spec_bins+1] energies at z = 0 and z = L */
  uint64_t* time_z;             /* [4][n_zbins] time per z segment, LSB 2^-50 s */
  uint64_t* time_r;             /* [4][n_rbins] time per radial bin, LSB 2^-50 s */
  uint64_t* cross_pos;          /* [4][n_zbins+1] crossings of z faces along +z */
  uint64_t* cross_neg;          /* [4][n_zbins+1] along -z */
  uint64_t* rcross_out;         /* [4][n_rbins+1] outward crossings of r = k R / n_rbins */
  uint64_t* rcross_in;          /* [4][n_rbins+1] inward crossings */
  uint64_t* wall;               /* [4][n_zbins] particles ended on the wall, by z segment */
  int64_t* ledger;              /* [ORC_OB_LEDGER_LEN] */
  double* energy;               /* [ORC_OE_LEN] */
  uint64_t* chan_count;         /* [n_channels] */
  uint64_t* per_primary;        /* [n] collisions in each primary's tree, may be NULL */
  double* end_state;            /* [n][8] x y z E ux uy uz t of each primary at its end, may be NULL */
} orc_orbit_tallies;

/* Raw tallies are ADDED to out.  Returns 0 on success, 1 for an invalid
 * problem or orbit, 2 for a channel kind the orbit mode does not take, 3 for
 * a primary outside the tube. */
int orc_orbit_run(const orc_problem* p, const orc_orbit* o, const orc_orbit_primaries* pr,
                  uint64_t seed, int n_threads, orc_orbit_tallies* out);

#ifdef __cplusplus
}
#endif
#endif
