// multi.cuh - device structures of the multi-request transport kernel.
//
// Many independent source configurations (requests) share one persistent
// launch.  Each request owns a slot: its parameter blocks for pass 1 and pass
// 2, its tally buffers, and a control line with the slot state and, per pass,
// one 64-bit word "generation | next primary | live particles".  Claims are a
// compare-and-swap on that word that never takes primaries past the end;
// products and deaths are single atomics on the live count, so a pass of a
// request is complete exactly when a decrement leaves no live particle with
// every primary claimed; the warp that observes it builds the request's
// target fields (pass 1 -> 2) or finalises and normalises its outputs (last
// pass) inside the kernel.
//
// A slot is reused by later requests.  The host gives each admission a new
// generation, carried in the state word (bits 8 and up) and, modulo 32, in the
// top bits of the pass words; a claim succeeds only on a word of the
// generation whose state the claiming lane read, so a lane delayed across a
// request's completion and the admission of the next request into its slot
// cannot take the new request's primaries under the old request's pass.
#pragma once
#include "karl_device.cuh"

namespace karl {

constexpr int MAX_SLOTS = 1024;          // request slots (10 bits in the particle word)
enum { SLOT_EMPTY = 0, SLOT_PASS1 = 1, SLOT_PASS2 = 2, SLOT_TRANS = 3, SLOT_DONE = 4 };

// pass word: generation (5 bits) | next primary (31 bits) | live particles (28 bits)
constexpr int WORD_NEXT_SHIFT = 28;
constexpr int WORD_GEN_SHIFT = 59;
constexpr unsigned long long WORD_LIVE_MASK = (1ULL << WORD_NEXT_SHIFT) - 1;
constexpr unsigned long long WORD_NEXT_MASK = (1ULL << (WORD_GEN_SHIFT - WORD_NEXT_SHIFT)) - 1;
constexpr long long MAX_REQUEST_PRIMARIES = (1LL << 31) - 1;

__host__ __device__ __forceinline__ unsigned long long word_gen(unsigned long long w) {
  return w >> WORD_GEN_SHIFT;
}
__host__ __device__ __forceinline__ long long word_next(unsigned long long w) {
  return (long long)((w >> WORD_NEXT_SHIFT) & WORD_NEXT_MASK);
}
__host__ __device__ __forceinline__ unsigned long long word_live(unsigned long long w) {
  return w & WORD_LIVE_MASK;
}
// slot state word: generation << 8 | SLOT_*
__host__ __device__ __forceinline__ int state_kind(int st) { return st & 0xff; }
__host__ __device__ __forceinline__ unsigned state_gen(int st) { return (unsigned)st >> 8; }

struct SlotCtl {
  unsigned long long word[2];            // per pass: generation | next primary | live
  int state;                             // generation << 8 | SLOT_*
  int pass;                              // pass being run (1 or 2)
  char pad[104];
};

struct SlotDesc {
  Params P[2];                           // pass-1 and pass-2 parameter blocks
  int n_passes;                          // 2 only when recombination channels exist
  int pad0;
  long long n_prim;
  unsigned long long* time1;             // [3][nz+2][ntb] pass-1 time (target fields)
  double* frate;                         // [nch][nz]
  double* fcol;                          // [nch][nz+1]
  unsigned long long* time_out;          // [3][nz+2][ntb] time of the last pass
  unsigned long long* cpos_out;          // [3][nz+1]
  unsigned long long* cneg_out;          // [3][nz+1]
  double* density;                       // [3][nz]
  double* current;                       // [3][nz+1]
  double* field;                         // [3][nz][ntb]
  double tsim, vol, area;
  const double* sig_cm;                  // channel-major cross sections (field builder)
  int* done_flag;                        // host-visible completion word (pinned, mapped)
  int pad1;
};

struct MultiCtl {
  Control c;                             // shared ring, abort, error, counters
  unsigned long long published;          // requests published by the host (sequence)
  char pad0[120];
  unsigned long long adopted;            // requests adopted by the kernel
  char pad1[120];
  unsigned long long done_count;
  char pad2[120];
  int shutdown;                          // host: leave once every published request is done
  int pad3;
  unsigned bitmap[MAX_SLOTS / 32];       // slots with unclaimed primaries in their pass
  unsigned pubq[MAX_SLOTS];              // slot of the request with sequence number q % MAX_SLOTS
};

}  // namespace karl
