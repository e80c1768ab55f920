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
#include "event.cuh"

namespace karl {

// ---------------------------------------------------------------------------
// persistent kernel

// Copy the column tables (and the pass-2 recombination fields) into dynamic
// shared memory when they fit; the event code reads them through P's pointers.
__device__ void stage_tables(Params& SP, const Params& Pk, double* dyn, int dyn_doubles) {
  const int nz = Pk.nz;
  int need = (4 * nz + 2) + (Pk.nq + 1 + 1) / 2 + 1;
  for (int k = 0; k < Pk.nch; ++k)
    if (Pk.fcol[k]) need += 2 * nz + 1;
  if (need > dyn_doubles) return;                   // stay in global memory
  double* col = dyn;
  double* fac = col + (nz + 1);
  double* nseg = fac + (nz + 1);
  double* invn = nseg + nz;
  int* ginv = (int*)(invn + nz);
  double* next = (double*)(ginv + ((Pk.nq + 2) & ~1));
  for (int i = threadIdx.x; i <= nz; i += blockDim.x) col[i] = Pk.colgas[i];
  for (int i = threadIdx.x; i <= nz; i += blockDim.x) fac[i] = Pk.faces[i];
  for (int i = threadIdx.x; i < nz; i += blockDim.x) nseg[i] = Pk.nseg[i];
  for (int i = threadIdx.x; i < nz; i += blockDim.x) invn[i] = Pk.invn[i];
  if (Pk.ginv)
    for (int i = threadIdx.x; i <= Pk.nq; i += blockDim.x) ginv[i] = Pk.ginv[i];
  if (threadIdx.x == 0) {
    SP.colgas = col;
    SP.faces = fac;
    SP.nseg = nseg;
    SP.invn = invn;
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
__global__ void __launch_bounds__(512, 1) transport_kernel(const Params Pk, Ring R, Control* ctl,
                                                        const volatile int* cancel,
                                                        unsigned long long timeout_ns,
                                                        int dyn_doubles) {
  const unsigned long long deadline = globaltimer_ns() + timeout_ns;
  if (threadIdx.x == 0 && ld_relaxed(&ctl->t_start) == 0)
    atomicCAS(&ctl->t_start, 0ULL, deadline - timeout_ns);
  // dynamic shared memory: the staged tables (dyn_doubles), then one product
  // queue and one batch of parked collisions per warp of the block
  extern __shared__ double dyn[];
  __shared__ Shared S;
  __shared__ Params SP;
  const int nwarps = blockDim.x >> 5;
  WarpQueue* wq = (WarpQueue*)(dyn + dyn_doubles);
  RareBuf* rbuf = (RareBuf*)(wq + nwarps);
  if (threadIdx.x == 0) SP = Pk;
  for (int i = threadIdx.x; i < LEDGER; i += blockDim.x) S.ledger[i] = 0;
  for (int i = threadIdx.x; i < MAXCH; i += blockDim.x) S.chan[i] = 0;
  if (threadIdx.x < nwarps) {
    wq[threadIdx.x].top = 0;
    rbuf[threadIdx.x].n = 0;
    rbuf[threadIdx.x].r = 0;
  }
  __syncthreads();
  stage_tables(SP, Pk, dyn, dyn_doubles);
  __syncthreads();
  const Params& P = SP;

  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  WarpQueue& Q = wq[threadIdx.x >> 5];
  RareBuf& Rb = rbuf[threadIdx.x >> 5];
  bool eager = false;
  bool has = false;
  Lane L;
  EventOut o;
  o.parked = false;
  o.flights = 0;
  o.colls = 0;
  o.recoil = 0;
  o.excit = 0;
  o.chan = -1;
  unsigned long long started = 0;
  unsigned long long idle_iters = 0, busy_iters = 0, busy_lane_iters = 0;
  unsigned idle_ns = 128;
  // A warp that still holds particles but found nothing for its idle lanes
  // skips its next refill attempts (1, 3, 7, ... up to 63 iterations): once
  // the primaries are used up, warps with a few long histories left would
  // otherwise contend for the ring head on every iteration.
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
      const unsigned long long pn = ld_relaxed(&ctl->prim_next);
      port.local = pn < (unsigned long long)P.n_prim;
      // The last primaries' histories set the end of the pass: from about two
      // primaries per lane before the end, parked collisions go at once so
      // those histories are not held up.
      eager = pn + 2ULL * gridDim.x * blockDim.x >= (unsigned long long)P.n_prim;
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
    unsigned need = __ballot_sync(FULL, !has);
    if (need && need != FULL && refill_skip > 0) {
      --refill_skip;
      need = 0;
    }
    if (need) {
      const int k = __popc(need);
      unsigned long long rbase = 0, pbase = 0;
      int rgot = 0, pgot = 0;
      if (lane == 0) {
        // Count the lanes as active only when work is visible, then claim it:
        // idle warps that find nothing leave the counter alone.  Lanes the
        // ring cannot fill take primaries in the same step -- also when a
        // contended claim on the ring fails -- unless the ring is three
        // quarters full (products first, so it cannot overflow).  Holding
        // lanes back for a ring only a quarter full left a quarter of the
        // FP32 form's lanes idle while every warp fought for the ring head.
        unsigned long long h = ld_relaxed(&ctl->head), t = ld_relaxed(&ctl->tail);
        const unsigned long long pn = ld_relaxed(&ctl->prim_next);
        const bool ring_work = h < t;
        const bool prim_work = pn < (unsigned long long)P.n_prim && t - h < R.cap / 4 * 3;
        if (ring_work || prim_work) {
          atomicAdd((unsigned long long*)&ctl->active, (unsigned long long)k);
          __threadfence();
          for (int tries = 0; tries < 16 && h < t; ++tries) {
            unsigned long long take = t - h < (unsigned long long)k ? t - h : (unsigned long long)k;
            unsigned long long old = atomicCAS(&ctl->head, h, h + take);
            if (old == h) { rbase = h; rgot = (int)take; break; }
            h = old;
            t = ld_relaxed(&ctl->tail);
          }
          if (rgot < k && prim_work) {
            const int want = k - rgot;
            unsigned long long p0 = atomicAdd(&ctl->prim_next, (unsigned long long)want);
            if (p0 < (unsigned long long)P.n_prim) {
              unsigned long long left = (unsigned long long)P.n_prim - p0;
              pbase = p0;
              pgot = left < (unsigned long long)want ? (int)left : want;
              if (left <= (unsigned long long)want) atomicMax(&ctl->t_claimed, globaltimer_ns());
            }
          }
          if (rgot + pgot < k)
            atomicAdd((unsigned long long*)&ctl->active, (unsigned long long)(rgot + pgot - k));
        }
      }
      rbase = __shfl_sync(FULL, rbase, 0);
      pbase = __shfl_sync(FULL, pbase, 0);
      rgot = __shfl_sync(FULL, rgot, 0);
      pgot = __shfl_sync(FULL, pgot, 0);
      if (rgot + pgot == 0) {
        refill_backoff = refill_backoff * 2 + 1;
        if (refill_backoff > 63) refill_backoff = 63;
        refill_skip = refill_backoff;
      } else {
        refill_backoff = 0;
      }
      bool born_dead = false;
      if (!has && rgot + pgot > 0) {
        const int rank = __popc(need & lt);
        if (rank < rgot + pgot) {
          if (rank < rgot) {
            has = ring_get(R, ctl, rbase + rank, L, deadline);
          } else {
            const unsigned long long idx = pbase + (rank - rgot);
            L.z = P.pz[idx];
            L.eq = quant_e(P.pe[idx]);
            L.mu = P.pmu[idx];
            L.sp = P.psp[idx];
            L.node = 0;
            L.tal = 0.0;
            L.ev = 0;
            L.pid = (unsigned long long)P.pid_offset + idx;
            L.j = segment_of(P, L.z);
            L.slot = 0;
            sadd(&S.ledger[L_E_IN_PRIMARY], L.eq);
            sadd(&S.ledger[L_BIRTHS + L.sp], 1);
            if (L.sp == SP_E && L.eq < P.ecut_q) {
              die<F32>(P, S.ledger, L, R_CUTOFF, L_E_CUTOFF);
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

    // ---- parked rare collisions: once enough have gathered, free lanes and
    // then busy ones -- whose particles wait in the slots the batch frees --
    // perform them together; near the end of the pass, at once ----
    __syncwarp();
    int rk = -1;
    const int nr = min(Rb.n, RB - Rb.r);
    const unsigned hm = __ballot_sync(FULL, has);
    const bool batch = nr >= RB_TRIGGER || (nr > 0 && (hm == 0 || eager));
    if (batch) {
      const int nfree = 32 - __popc(hm);
      const int rank = has ? nfree + __popc(hm & lt) : __popc(~hm & lt);
      const bool take = rank < nr;
      const bool give = take && has;
      Lane back;
      if (give) {
        back = L;
      }
      if (take) {
        L = Rb.s[nr - 1 - rank];
        rk = Rb.ch[nr - 1 - rank];
        has = true;
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
    if (has && rk >= 0) {
      unsigned long long w[4];
      parked_block(P, L, w);
      o.alive = true;
      o.parked = false;
      o.chan = -1;
      rare_kinematics<F32>(P, S.ledger, L, o, port, rk, w);
      if (!o.alive) { has = false; died = true; }
    } else if (has) {
      event<F32>(P, S.ledger, L, o, port);
      if (!o.alive) { has = false; died = !o.parked; }
    }
    __syncwarp();
    if (lane == 0) {
      if (Q.top > WQ) Q.top = WQ;                     // pushes past the end went to the ring
      if (Rb.n > RB - Rb.r) Rb.n = RB - Rb.r;         // parks past the end were done in line
    }

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
    atomicMax(&ctl->t_end, globaltimer_ns());
    atomicAdd(&ctl->idle_iters, idle_iters);
    atomicAdd(&ctl->spilled, sp);
    atomicAdd(&ctl->busy_iters, busy_iters);
    atomicAdd(&ctl->busy_lane_iters, busy_lane_iters);
    atomicAdd(&S.ledger[L_N_FLIGHT], f);
    atomicAdd(&S.ledger[L_N_COLL], c);
    atomicAdd(&S.ledger[L_N_FLIGHT_ALL], f);
    atomicAdd(&S.ledger[L_N_COLL_ALL], c);
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

// dynamic shared memory for the staged tables: at most this much per block,
// so that two blocks of 256 threads (with ~33 KB more for their warp queues
// and parked collisions) still fit one SM's 227 KB; blocks of 128 threads
// need half the queue memory and fit four to an SM with config-sized tables
constexpr int DYN_MAX_BYTES = 76 * 1024;
// per-warp queues in dynamic shared memory (after the tables)
constexpr int QUEUE_BYTES_PER_WARP = (int)(sizeof(WarpQueue) + sizeof(RareBuf));
static_assert(sizeof(WarpQueue) % 8 == 0 && sizeof(RareBuf) % 8 == 0, "queue alignment");


// Shared memory a block may give its staged tables: 76 KB for blocks of up
// to 256 threads (two to an SM), and what a block of more threads, alone on
// its SM, leaves beside its queues (then the pass-2 field tables fit too).
constexpr int SMEM_PER_SM = 227 * 1024;
constexpr int STATIC_SMEM_MARGIN = 4 * 1024;
int dyn_table_budget(int block) {
  if (block <= 256) return DYN_MAX_BYTES;
  return SMEM_PER_SM - STATIC_SMEM_MARGIN - (block / 32) * QUEUE_BYTES_PER_WARP;
}

// Doubles of dynamic shared memory the staged tables of P need (0: too big,
// read them from global memory).
int transport_dyn_doubles(const Params& P, int block) {
  int need = (4 * P.nz + 2) + (P.nq + 1 + 1) / 2 + 1;
  for (int k = 0; k < P.nch; ++k)
    if (P.fcol[k]) need += 2 * P.nz + 1;
  return need * 8 <= dyn_table_budget(block) ? need : 0;
}

size_t transport_dyn_bytes(const Params& P, int block) {
  return (size_t)transport_dyn_doubles(P, block) * 8 + (size_t)(block / 32) * QUEUE_BYTES_PER_WARP;
}

cudaError_t launch_transport(bool f32, const Params& P, const Ring& R, Control* ctl,
                             const volatile int* cancel, unsigned long long timeout_ns, int grid,
                             int block, cudaStream_t st) {
  const int dd = transport_dyn_doubles(P, block);
  const size_t bytes = transport_dyn_bytes(P, block);
  if (f32)
    transport_kernel<true><<<grid, block, bytes, st>>>(P, R, ctl, cancel, timeout_ns, dd);
  else
    transport_kernel<false><<<grid, block, bytes, st>>>(P, R, ctl, cancel, timeout_ns, dd);
  return cudaGetLastError();
}

cudaError_t transport_setup() {
  cudaError_t e = cudaFuncSetAttribute(transport_kernel<true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       SMEM_PER_SM - STATIC_SMEM_MARGIN);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(transport_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              SMEM_PER_SM - STATIC_SMEM_MARGIN);
}

cudaError_t transport_occupancy(bool f32, const Params& P, int block, int* blocks_per_sm) {
  const size_t bytes = transport_dyn_bytes(P, block);
  if (f32)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, transport_kernel<true>,
                                                         block, bytes);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, transport_kernel<false>,
                                                       block, bytes);
}

}  // namespace karl
