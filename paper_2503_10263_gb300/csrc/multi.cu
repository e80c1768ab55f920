// multi.cu - persistent transport kernel over many requests (batched and
// served forms of the transport step).
//
// The event itself is the same as in the single-run kernel (event.cuh).  What
// differs is where work comes from and where it goes: every particle carries
// its request slot; idle lanes take their warp's products, then products from
// the shared ring, then primaries of any request whose current pass still has
// unclaimed primaries (a bitmap of slots); each request moves pass 1 ->
// target fields -> pass 2 -> final tallies inside the kernel, driven by the
// warp whose atomic decrement emptied the request's pass.  A batch is a launch
// with every request published before it starts; a server keeps the launch
// running while the host publishes requests into free slots.
#include "event.cuh"
#include "multi.cuh"

namespace karl {

__device__ __forceinline__ int ld_acquire_i(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_i(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// cross section from the channel-major table (target-field builder)
__device__ double sigma_cm(const double* sig, int n, double e_min, double log_ratio_h, double loss,
                           double e) {
  if (!(e > loss)) return 0.0;
  double x = log(e / e_min) / log_ratio_h;
  int i = (int)floor(x);
  double f;
  if (i < 0) { i = 0; f = 0.0; }
  else if (i > n - 2) { i = n - 2; f = 1.0; }
  else f = x - (double)i;
  return (1.0 - f) * sig[i] + f * sig[i + 1];
}

// Warp-cooperative end of pass p of request s (Eq. target_field_density for
// the fields; Sec. 2.3 for the current).
__device__ void complete_pass(SlotDesc* D, SlotCtl* C, MultiCtl* M, int s, int p, int lane) {
  // the request is alive until this completes, so its generation is current
  int ok = 0, gen_bits = 0;
  if (lane == 0) {
    gen_bits = ld_acquire_i(&C[s].state) & ~0xff;
    const int from = gen_bits | (p == 1 ? SLOT_PASS1 : SLOT_PASS2);
    ok = atomicCAS(&C[s].state, from, gen_bits | SLOT_TRANS) == from;
  }
  gen_bits = __shfl_sync(FULL, gen_bits, 0);
  if (!__shfl_sync(FULL, ok, 0)) return;                 // someone else already did it
  SlotDesc& d = D[s];
  const Params& P = d.P[p - 1];
  const int nz = P.nz, ntb = P.ntb;
  const double inv_qt = 1.0 / Q_T;
  if (p == 1 && d.n_passes == 2) {
    // pass-1 time: point adds plus the prefix of the range adds
    for (int col = lane; col < NSP * ntb; col += 32) {
      const int sp = col / ntb, b = col % ntb;
      unsigned long long acc = 0;
      for (int row = 0; row < nz + 2; ++row) {
        const size_t i = ((size_t)sp * (nz + 2) + row) * ntb + b;
        acc += P.time_rg[i];
        d.time1[i] = P.time_pt[i] + acc;
      }
    }
    __syncwarp();
    __threadfence();
    // target fields of the recombination channels
    for (int t = lane; t < P.nch * nz; t += 32) {
      const int k = t / nz, j = t % nz;
      const ChanDev& ch = P.ch[k];
      if (ch.kind != RECOMBINATION) continue;
      double acc = 0.0;
      for (int b = 0; b < ntb; ++b) {
        const unsigned long long tt = d.time1[((size_t)ch.sout * (nz + 2) + (j + 1)) * ntb + b];
        const double n = (double)tt * inv_qt / (d.tsim * d.vol);
        if (ch.sin == SP_E) {
          acc += n;
        } else {
          const double eb = P.e_min * exp(P.log_ratio_h * (P.n_energy - 1) * (b + 0.5) / ntb);
          const double x = eb * P.inv_mass[SP_E];
          const double v = C_LIGHT * sqrt(x * (2.0 + x)) / (1.0 + x);
          acc += n * sigma_cm(d.sig_cm + (size_t)k * P.n_energy, P.n_energy, P.e_min,
                              P.log_ratio_h, ch.loss_ev, eb) * v;
        }
      }
      d.frate[(size_t)k * nz + j] = acc;
    }
    __syncwarp();
    __threadfence();
    for (int k = lane; k < P.nch; k += 32) {
      if (P.ch[k].kind != RECOMBINATION) continue;
      double c = 0.0;
      d.fcol[(size_t)k * (nz + 1)] = 0.0;
      for (int j = 0; j < nz; ++j) {
        c += d.frate[(size_t)k * nz + j] * P.dz;
        d.fcol[(size_t)k * (nz + 1) + j + 1] = c;
      }
    }
    __syncwarp();
    __threadfence();
    if (lane == 0) {
      *(volatile int*)&C[s].pass = 2;
      __threadfence();
      st_release_i(&C[s].state, gen_bits | SLOT_PASS2);
      if (d.n_prim > 0) atomicOr(&M->bitmap[s >> 5], 1u << (s & 31));
    }
    return;
  }
  // last pass: prefix sums into the outputs, then normalise
  for (int col = lane; col < NSP * ntb; col += 32) {
    const int sp = col / ntb, b = col % ntb;
    unsigned long long acc = 0;
    for (int row = 0; row < nz + 2; ++row) {
      const size_t i = ((size_t)sp * (nz + 2) + row) * ntb + b;
      acc += P.time_rg[i];
      d.time_out[i] = P.time_pt[i] + acc;
    }
  }
  for (int sp = lane; sp < 2 * NSP; sp += 32) {
    const unsigned long long* rg = sp < NSP ? P.xpos_rg : P.xneg_rg;
    unsigned long long* out = sp < NSP ? d.cpos_out : d.cneg_out;
    const int ss = sp % NSP;
    unsigned long long acc = 0;
    for (int k = 0; k <= nz; ++k) {
      acc += rg[(size_t)ss * (nz + 2) + k];
      out[(size_t)ss * (nz + 1) + k] = acc;
    }
  }
  __syncwarp();
  __threadfence();
  const unsigned long long* t1 = d.n_passes == 2 ? d.time1 : d.time_out;
  for (int t = lane; t < NSP * nz; t += 32) {
    const int sp = t / nz, j = t % nz;
    double tsum = 0.0;
    for (int b = 0; b < ntb; ++b) {
      const size_t idx = ((size_t)sp * (nz + 2) + (j + 1)) * ntb + b;
      tsum += (double)d.time_out[idx] * inv_qt;
      d.field[((size_t)sp * nz + j) * ntb + b] = (double)t1[idx] * inv_qt / (d.tsim * d.vol);
    }
    d.density[(size_t)sp * nz + j] =
        tsum / (d.tsim * d.vol) - (double)P.recomb[(size_t)sp * nz + j] / d.vol;
  }
  for (int t = lane; t < NSP * (nz + 1); t += 32)
    d.current[t] = ((double)d.cpos_out[t] - (double)d.cneg_out[t]) / (d.area * d.tsim);
  __syncwarp();
  __threadfence_system();
  if (lane == 0) {
    st_release_i(&C[s].state, gen_bits | SLOT_DONE);
    atomicAdd(&M->done_count, 1ULL);
    *(volatile int*)d.done_flag = 1;
    __threadfence_system();
  }
}

// A pass of request s empties when a decrement of its word leaves no live
// particle and every primary claimed.
__device__ __forceinline__ bool pass_emptied(unsigned long long old, unsigned long long dec,
                                             long long n_prim) {
  return word_live(old) == dec && word_next(old) >= n_prim;
}

// Claim up to k primaries of the current pass of the request in slot s, whose
// state the caller read as st (a pass state).  The claim is a compare-and-swap
// on the pass word that adds the same count to the next primary and to the
// live particles, only while the word carries the generation of st and
// primaries remain, so it never takes primaries past the end and never
// touches a later request in the slot.  Returns the count claimed (0 if
// none) and the first index; clears the slot's bit when it takes the last.
__device__ __forceinline__ int claim_primaries(SlotDesc* D, SlotCtl* C, MultiCtl* M, int s, int st,
                                               int k, unsigned long long* first) {
  const int p = state_kind(st) == SLOT_PASS2 ? 2 : 1;
  unsigned long long* word = &C[s].word[p - 1];
  // the descriptor of the generation read in st (admission writes the new
  // generation's pass words before its descriptor, so a newer descriptor
  // comes with a newer word, which the generation test below rejects)
  const long long n = (long long)ld_acquire((const unsigned long long*)&D[s].n_prim);
  const unsigned long long gen = (unsigned long long)(state_gen(st) & 31u);
  unsigned long long old = ld_acquire(word);
  for (int tries = 0; tries < 64; ++tries) {
    if (word_gen(old) != gen) return 0;               // the slot holds another request now
    const long long next = word_next(old);
    const long long left = n - next;
    if (left <= 0) return 0;                          // every primary of this pass claimed
    const int g = left < k ? (int)left : k;
    const unsigned long long nw =
        old + ((unsigned long long)g << WORD_NEXT_SHIFT) + (unsigned long long)g;
    const unsigned long long prev = atomicCAS(word, old, nw);
    if (prev == old) {
      if (next + g >= n) atomicAnd(&M->bitmap[s >> 5], ~(1u << (s & 31)));
      *first = (unsigned long long)next;
      return g;
    }
    old = prev;
  }
  return 0;                                           // contended: look elsewhere
}

template <bool F32>
__global__ void __launch_bounds__(256, 2) multi_kernel(SlotDesc* D, SlotCtl* C, MultiCtl* M, Ring R,
                                                    const volatile int* cancel,
                                                    unsigned long long timeout_ns) {
  const unsigned long long deadline = globaltimer_ns() + timeout_ns;
  __shared__ WarpQueue wq[WARPS];
  __shared__ RareBuf rbuf[WARPS];
  if (threadIdx.x < WARPS) {
    wq[threadIdx.x].top = 0;
    rbuf[threadIdx.x].n = 0;
    rbuf[threadIdx.x].r = 0;
  }
  __syncthreads();
  Control* ctl = &M->c;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  WarpQueue& Q = wq[threadIdx.x >> 5];
  RareBuf& Rb = rbuf[threadIdx.x >> 5];
  bool has = false;
  Lane L;
  L.slot = 0;
  int lpass = 1;
  const Params* Pl = &D[0].P[0];
  EventOut o;
  o.flights = o.colls = o.recoil = o.excit = 0;
  o.chan = -1;
  o.parked = false;
  unsigned long long idle_iters = 0, busy_iters = 0, busy_lane_iters = 0, started = 0;
  unsigned idle_ns = 128;
  // a warp that holds particles but found nothing for its idle lanes skips
  // its next refill attempts (1, 3, 7, ... up to 63 iterations)
  int refill_skip = 0, refill_backoff = 0;
  RingPort port;
  port.R = &R;
  port.ctl = ctl;
  port.deadline = deadline;
  port.q = &Q;
  port.rare = &Rb;
  port.local = true;
  port.spilled = 0;
  port.slot_live = nullptr;

  // the lane's particle belongs to the current pass of its request
  auto bind = [&](int s) {
    lpass = ld_acquire_i(&C[s].pass);
    lpass = lpass == 2 ? 2 : 1;
    Pl = &D[s].P[lpass - 1];
  };
  // per-lane sums belong to the request of the lane's particle: they go to
  // its ledger whenever the lane lets the particle go (death, park, hand-back)
  auto flush_sums = [&]() {
    unsigned long long* led = Pl->ledger;
    if (o.flights) {
      atomicAdd(led + L_N_FLIGHT, o.flights);
      atomicAdd(led + L_N_FLIGHT_ALL, o.flights);
    }
    if (o.colls) {
      atomicAdd(led + L_N_COLL, o.colls);
      atomicAdd(led + L_N_COLL_ALL, o.colls);
    }
    if (o.recoil) atomicAdd(led + L_LOSS_RECOIL, o.recoil);
    if (o.excit) atomicAdd(led + L_LOSS_EXCIT, o.excit);
    o.flights = o.colls = o.recoil = o.excit = 0;
  };
  // a pass this lane saw empty (by the death of a particle or a primary born dead)
  int trigB = 0, tslotB = 0, tpassB = 1;

  for (long long iter = 0;; ++iter) {
    if ((iter & 63) == 0) {
      int stop = 0, local = 0;
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
        // adopt requests the host has published since the last look
        unsigned long long pub = ld_acquire(&M->published);
        unsigned long long ad = ld_relaxed(&M->adopted);
        while (ad < pub) {
          const unsigned long long old = atomicCAS(&M->adopted, ad, ad + 1);
          if (old == ad) {
            const int s = (int)ld_acquire_i((const int*)&M->pubq[ad % MAX_SLOTS]);
            // (requests without primaries are finished by the host, never published)
            if (state_kind(ld_acquire_i(&C[s].state)) == SLOT_PASS1)
              atomicOr(&M->bitmap[s >> 5], 1u << (s & 31));
            ++ad;
          } else {
            ad = old;
          }
        }
        for (int i = 0; i < MAX_SLOTS / 32 && !local; ++i)
          local = ld_relaxed_i((const int*)&M->bitmap[i]) != 0;
      }
      if (__shfl_sync(FULL, stop, 0)) break;
      port.local = __shfl_sync(FULL, local, 0) != 0;
    }

    // ---- idle lanes first resume particles handed back for a batch ----
    __syncwarp();
    if (Rb.r > 0) {
      const unsigned needr = __ballot_sync(FULL, !has);
      const int r0 = Rb.r;
      const int tr = min(__popc(needr), r0);
      if (!has) {
        const int rank = __popc(needr & lt);
        if (rank < tr) {
          L = Rb.s[RB - r0 + rank];
          has = true;
          bind(L.slot);
        }
      }
      __syncwarp();
      if (lane == 0) Rb.r = r0 - tr;
      __syncwarp();
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
          bind(L.slot);
        }
      }
      int left = top - take;
      if (!port.local && left > 0) {
        unsigned long long pos = 0;
        if (lane == 0) pos = atomicAdd(&ctl->tail, (unsigned long long)left);
        pos = __shfl_sync(FULL, pos, 0);
        if (lane < left) ring_put(R, ctl, pos + lane, Q.s[lane], deadline);
        if (lane == 0) port.spilled += left;
        left = 0;
      }
      __syncwarp();
      if (lane == 0) Q.top = left;
      __syncwarp();
    }

    // ---- other idle lanes: products from the ring, then primaries of a request ----
    unsigned need = __ballot_sync(FULL, !has);
    if (need && need != FULL && refill_skip > 0) {
      --refill_skip;
      need = 0;
    }
    if (need) {
      const int k = __popc(need);
      unsigned long long base = 0;
      int got = 0, src = 0, gslot = 0, gpass = 1;
      if (lane == 0) {
        unsigned long long h = ld_relaxed(&ctl->head), t = ld_relaxed(&ctl->tail);
        for (int tries = 0; tries < 16 && h < t; ++tries) {
          unsigned long long take = t - h < (unsigned long long)k ? t - h : (unsigned long long)k;
          unsigned long long old = atomicCAS(&ctl->head, h, h + take);
          if (old == h) { base = h; got = (int)take; src = 1; break; }
          h = old;
          t = ld_relaxed(&ctl->tail);
        }
        if (got == 0) {
          // A request with unclaimed primaries.  The search starts at a slot
          // chosen by the block, so the warps of a block keep to one request
          // while it lasts and its parameters and column tables stay in L1.
          const unsigned long long pub = ld_relaxed(&M->published);
          const unsigned long long dn = ld_relaxed(&M->done_count);
          const unsigned long long act = pub > dn ? pub - dn : 1ULL;
          const int s0 = (int)((unsigned long long)blockIdx.x % (act < MAX_SLOTS ? act : MAX_SLOTS));
          for (int i = 0; i <= MAX_SLOTS / 32 && got == 0; ++i) {
            const int wi = ((s0 >> 5) + i) & (MAX_SLOTS / 32 - 1);
            unsigned bits = (unsigned)ld_relaxed_i((const int*)&M->bitmap[wi]);
            if (i == 0) bits &= ~0u << (s0 & 31);                       // from s0 on
            else if (i == MAX_SLOTS / 32) bits &= ~(~0u << (s0 & 31));  // wrapped: below s0
            while (bits && got == 0) {
              const int bit = __ffs(bits) - 1;
              bits &= bits - 1;
              const int s = wi * 32 + bit;
              const int st = ld_acquire_i(&C[s].state);
              if (state_kind(st) != SLOT_PASS1 && state_kind(st) != SLOT_PASS2) continue;
              // Only the claim that takes the last primaries clears the bit; a
              // claim on a pass that has ended takes nothing and leaves the bit
              // alone (the warp completing pass 1 sets it again for pass 2).
              // The taking claim holds live particles, so the pass cannot end
              // before its clear.
              unsigned long long first = 0;
              const int g = claim_primaries(D, C, M, s, st, k, &first);
              if (g > 0) {
                got = g;
                base = first;
                src = 2;
                gslot = s;
                gpass = state_kind(st) == SLOT_PASS2 ? 2 : 1;
              }
            }
          }
        }
      }
      base = __shfl_sync(FULL, base, 0);
      got = __shfl_sync(FULL, got, 0);
      src = __shfl_sync(FULL, src, 0);
      gslot = __shfl_sync(FULL, gslot, 0);
      gpass = __shfl_sync(FULL, gpass, 0);
      if (got == 0) {
        refill_backoff = refill_backoff * 2 + 1;
        if (refill_backoff > 63) refill_backoff = 63;
        refill_skip = refill_backoff;
      } else {
        refill_backoff = 0;
      }
      if (!has && got > 0) {
        const int rank = __popc(need & lt);
        if (rank < got) {
          const unsigned long long idx = base + rank;
          if (src == 1) {
            has = ring_get(R, ctl, idx, L, deadline);
            if (has) bind(L.slot);
          } else {
            lpass = gpass;
            Pl = &D[gslot].P[gpass - 1];
            const Params& P = *Pl;
            L.z = P.pz[idx];
            L.eq = quant_e(P.pe[idx]);
            L.mu = P.pmu[idx];
            L.sp = P.psp[idx];
            L.node = 0;
            L.tal = 0.0;
            L.ev = 0;
            L.pid = (unsigned long long)P.pid_offset + idx;
            L.j = segment_of(P, L.z);
            L.slot = gslot;
            sadd(P.ledger + L_E_IN_PRIMARY, L.eq);
            sadd(P.ledger + L_BIRTHS + L.sp, 1);
            if (L.sp == SP_E && L.eq < P.ecut_q) {
              die<F32>(P, P.ledger, L, R_CUTOFF, L_E_CUTOFF);
              const unsigned long long o2 =
                  atomicAdd(&C[gslot].word[gpass - 1], (unsigned long long)0 - 1ULL);
              if (pass_emptied(o2, 1ULL, D[gslot].n_prim)) { trigB = 1; tslotB = gslot; tpassB = gpass; }
            } else {
              has = true;
            }
          }
          started += 1;
        }
      }
    }

    // ---- parked rare collisions: once enough have gathered, free lanes and
    // then busy ones -- whose particles wait in the slots the batch frees --
    // perform them together.  When the primaries are used up the products of
    // parked collisions may be the work that is left, so they go at once ----
    __syncwarp();
    int rk = -1;
    const int nr = min(Rb.n, RB - Rb.r);
    const unsigned hm = __ballot_sync(FULL, has);
    const bool batch = nr >= RB_TRIGGER || (nr > 0 && (hm == 0 || !port.local));
    if (batch) {
      const int nfree = 32 - __popc(hm);
      const int rank = has ? nfree + __popc(hm & lt) : __popc(~hm & lt);
      const bool take = rank < nr;
      const bool give = take && has;
      Lane back;
      if (give) {
        flush_sums();                              // the lane changes particle
        back = L;
      }
      if (take) {
        L = Rb.s[nr - 1 - rank];
        rk = Rb.ch[nr - 1 - rank];
        has = true;
        bind(L.slot);
      }
      __syncwarp();                                // every parked slot has been read
      const int r0 = Rb.r;
      if (give) Rb.s[RB - r0 - 1 - (rank - nfree)] = back;   // stays counted as live
      __syncwarp();
      if (lane == 0) {
        Rb.r = r0 + max(nr - nfree, 0);
        Rb.n = 0;
      }
      __syncwarp();
    }

    // ---- one event ----
    bool died = false;
    const unsigned busy = __ballot_sync(FULL, has);
    if (busy) {
      idle_ns = 128;
      busy_lane_iters += __popc(busy);
      ++busy_iters;
      if (has && rk >= 0) {
        port.slot_live = &C[L.slot].word[lpass - 1];
        unsigned long long w[4];
        parked_block(*Pl, L, w);
        o.alive = true;
        o.parked = false;
        o.chan = -1;
        rare_kinematics<F32>(*Pl, Pl->ledger, L, o, port, rk, w);
        if (!o.alive) { has = false; died = true; }
      } else if (has) {
        port.slot_live = &C[L.slot].word[lpass - 1];
        event<F32>(*Pl, Pl->ledger, L, o, port);
        if (!o.alive) {
          has = false;
          died = !o.parked;
          if (o.parked) flush_sums();
        }
      }
      __syncwarp();
      if (lane == 0) {
        if (Q.top > WQ) Q.top = WQ;
        if (Rb.n > RB - Rb.r) Rb.n = RB - Rb.r;
      }
      // channel counts, one add per distinct (request, channel) per warp
      const unsigned mc = __ballot_sync(FULL, o.chan >= 0);
      if (o.chan >= 0) {
        const unsigned key = ((unsigned)L.slot << 5) | (unsigned)o.chan;
        const unsigned grp = __match_any_sync(mc, key);
        if (lane == __ffs(grp) - 1)
          atomicAdd(Pl->chan_count + o.chan, (unsigned long long)__popc(grp));
      }
      o.chan = -1;
      if (died) {
        flush_sums();
        const unsigned long long o2 =
            atomicAdd(&C[L.slot].word[lpass - 1], (unsigned long long)0 - 1ULL);
        if (pass_emptied(o2, 1ULL, D[L.slot].n_prim)) { trigB = 1; tslotB = L.slot; tpassB = lpass; }
      }
    }

    // ---- passes that just emptied: the whole warp finishes them ----
    {
      unsigned mt = __ballot_sync(FULL, trigB);
      while (mt) {
        const int srcl = __ffs(mt) - 1;
        const int s = __shfl_sync(FULL, tslotB, srcl);
        const int p = __shfl_sync(FULL, tpassB, srcl);
        complete_pass(D, C, M, s, p, lane);
        mt &= mt - 1;
      }
    }
    trigB = 0;

    if (!busy) {
      // leave when the host has closed the session and every published
      // request is done
      int done = 0;
      if (lane == 0) {
        done = ld_relaxed_i(&M->shutdown) &&
               ld_relaxed(&M->done_count) >= ld_acquire(&M->published);
      }
      if (__shfl_sync(FULL, done, 0)) break;
      __nanosleep(idle_ns);
      if (idle_ns < 8192) idle_ns <<= 1;
      ++idle_iters;
    }
  }

  unsigned long long sp = port.spilled, st = started;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    sp += __shfl_down_sync(FULL, sp, off);
    st += __shfl_down_sync(FULL, st, off);
  }
  if (lane == 0) {
    atomicAdd(&ctl->idle_iters, idle_iters);
    atomicAdd(&ctl->busy_iters, busy_iters);
    atomicAdd(&ctl->busy_lane_iters, busy_lane_iters);
    atomicAdd(&ctl->spilled, sp);
    atomicAdd(&ctl->particles, st);
  }
}

cudaError_t launch_multi(bool f32, SlotDesc* D, SlotCtl* C, MultiCtl* M, const Ring& R,
                         const volatile int* cancel, unsigned long long timeout_ns, int grid,
                         int block, cudaStream_t st) {
  if (f32)
    multi_kernel<true><<<grid, block, 0, st>>>(D, C, M, R, cancel, timeout_ns);
  else
    multi_kernel<false><<<grid, block, 0, st>>>(D, C, M, R, cancel, timeout_ns);
  return cudaGetLastError();
}

cudaError_t multi_occupancy(bool f32, int block, int* blocks_per_sm) {
  if (f32)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, multi_kernel<true>, block, 0);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, multi_kernel<false>, block, 0);
}

}  // namespace karl
