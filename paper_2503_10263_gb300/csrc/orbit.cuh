// orbit.cuh - device structures of the full-orbit transport (the Boris mover
// of Sec. 3.1) in a beam tube.
//
// Each particle carries its position (x, y, z) and proper velocity
// u = gamma v; every step is one relativistic Boris push in the uniform
// magnetic field B along +z and the electric field
// E = (e_r x, e_r y, E_z[segment of z]).  A flight ends where the optical
// depth summed over its steps reaches -ln(eta), at z = 0 or L, on the tube
// wall r = R, or at the lifetime cap.  Products of a generation go to the
// next generation's list; the host launches one kernel per generation.
#pragma once
#include "karl_device.cuh"

namespace karl {

// integer ledger of an orbit run
enum { OB_BIRTHS = 0, OB_DEATHS = 4, OB_N_COLL = 36, OB_N_FLIGHT = 37, OB_N_STEP = 38,
       OB_N_SPAWN_E = 39, OB_N_SPAWN_ION = 40, OB_LEDGER = 48 };
// death reasons
enum { OR_EXIT0 = 0, OR_EXIT1 = 1, OR_WALL = 2, OR_CUTOFF = 3, OR_CAP_COLL = 4,
       OR_CAP_TIME = 5, OR_CLUSTER = 6, OR_STALLED = 7 };
// energy ledger (eV)
enum { OE_IN_PRIMARY = 0, OE_IN_THERMAL = 1, OE_EXIT0 = 2, OE_EXIT1 = 3, OE_WALL = 4,
       OE_CUTOFF = 5, OE_CAP = 6, OE_CLUSTER = 7, OE_LOSS_IONIZ = 8, OE_LOSS_EXCIT = 9,
       OE_RECOIL = 10, OE_STALLED = 11, OE_FIELD_WORK = 12, OE_LEN = 16 };

// Particles of one generation (structure of arrays).
struct OrbitList {
  double* x;
  double* y;
  double* z;
  double* ux;
  double* uy;
  double* uz;
  unsigned long long* node;
  unsigned long long* pid;
  uint8_t* sp;
};

struct OrbitDev {
  double bz;                    // magnetic field along +z (T)
  double R2;                    // wall radius squared
  double r_scale;               // radial bins per metre (first guess of a bin)
  const double* edge2;          // [nr+1] squared radii of the radial bin edges
  double er;                    // radial field per metre (V/m^2)
  double dt[NSP];               // Boris time step per species
  double h[NSP];                // q dt / 2m per species (m/s per V/m)
  double e_cut, spec_bin;       // energies in eV
  double inv_dz;                // n_zbins / L (segment of z: floor(z inv_dz))
  double e_max;                 // top of the energy grid (eV)
  const double* u2edge;         // [4][n_tebins+1] u^2 at the energy-bin edges
  const double* ez;             // [nz] axial field per segment (V/m), NULL: none
  int nr;                       // radial bins
  int fields;                   // an electric field is present
  unsigned long long max_steps; // steps per flight before "stalled"
  // source of this generation: the primaries, or the list `in`
  int from_primaries;
  long long n_in;
  const double* px;
  const double* py;
  const double* pz;
  const double* pe;
  const double* pmu;
  const double* pphi;
  const uint8_t* psp;
  OrbitList in, out;
  unsigned long long out_cap;
  unsigned long long* counters; // [0] next particle to claim, [1] products written
  // raw tallies
  unsigned long long* time_z;   // [4][nz]
  unsigned long long* time_r;   // [4][nr]
  unsigned long long* xpos;     // [4][nz+1]
  unsigned long long* xneg;     // [4][nz+1]
  unsigned long long* rout;     // [4][nr+1]
  unsigned long long* rin;      // [4][nr+1]
  unsigned long long* wall;     // [4][nz]
  unsigned long long* spectrum; // [2][4][nspec+1]
  unsigned long long* ledger;   // [OB_LEDGER]
  unsigned long long* chan;     // [nch]
  unsigned long long* per_primary;  // [n primaries] or NULL
  double* energy;               // [OE_LEN]
  double* end_state;            // [n primaries][8] or NULL
  // limits
  int* error;                   // ERR_* of the launch
  const volatile int* cancel;
  unsigned long long timeout_ns; // time limit of one launch
};

}  // namespace karl
