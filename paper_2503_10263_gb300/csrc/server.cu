// server.cu - batched and served forms of the transport step (C ABI in
// include/karl.h, karl_server_*).
//
// Host side of the multi-request kernel (multi.cu): request records, a
// first-fit arena over one device allocation (admission by HBM footprint),
// publication of admitted requests into the running launch through a small
// queue in device memory, and collection of finished requests into the
// caller's buffers while the launch keeps running.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "host_common.h"
#include "multi.cuh"

namespace karl {
cudaError_t launch_multi(bool f32, SlotDesc* D, SlotCtl* C, MultiCtl* M, const Ring& R,
                         const volatile int* cancel, unsigned long long timeout_ns, int grid,
                         int block, cudaStream_t st);
cudaError_t multi_occupancy(bool f32, int block, int* blocks_per_sm);
}  // namespace karl

using namespace karl;

namespace {

constexpr size_t ALIGN = 256;
size_t up(size_t n) { return (n + ALIGN - 1) / ALIGN * ALIGN; }

// first-fit allocator over [0, size)
struct Arena {
  size_t size = 0, in_use = 0, peak = 0;
  std::map<size_t, size_t> free_;              // offset -> length
  void init(size_t n) {
    size = n;
    free_.clear();
    free_[0] = n;
    in_use = peak = 0;
  }
  bool alloc(size_t n, size_t* off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < n) continue;
      *off = it->first;
      const size_t rest = it->second - n, at = it->first + n;
      free_.erase(it);
      if (rest) free_[at] = rest;
      in_use += n;
      peak = std::max(peak, in_use);
      return true;
    }
    return false;
  }
  void release(size_t off, size_t n) {
    in_use -= n;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

// element counts of one request's arrays
struct Sizes {
  size_t n, nz, ntb, nt, nspec, cross_rg, cross, rec, nch, nq;
  explicit Sizes(const karl_geometry& g, size_t n_prim, int nch_, int nq_) {
    n = n_prim;
    nz = (size_t)g.n_zbins;
    ntb = (size_t)g.n_tebins;
    nt = (size_t)NSP * (nz + 2) * ntb;
    nspec = (size_t)2 * NSP * (g.n_spec_bins + 1);
    cross_rg = (size_t)NSP * (nz + 2);
    cross = (size_t)NSP * (nz + 1);
    rec = (size_t)NSP * nz;
    nch = (size_t)std::max(nch_, 1);
    nq = (size_t)nq_;
  }
};

enum { REQ_QUEUED = 0, REQ_ADMITTED = 1, REQ_FINISHED = 2, REQ_FAILED = 3 };

struct Request {
  uint64_t id = 0;
  int state = REQ_QUEUED;
  int slot = -1;
  size_t off = 0, bytes = 0;
  karl_geometry g;
  std::vector<double> nseg, z, e, mu;
  std::vector<uint8_t> sp;
  int64_t n_decays = 0, pid_offset = 0;
  uint64_t seed = 0;
  int n_passes = 1;
  karl_tallies out;
  ColumnTables tabs;
  std::vector<double> n2, col2;      // three-body clustering field (empty if unused)
  // device pointers of the final pass and of the outputs, for collection
  unsigned long long *spec = nullptr, *rec = nullptr, *led = nullptr, *chan = nullptr;
  unsigned long long* led1 = nullptr;   // pass-1 ledger of a two-pass request, else NULL
  unsigned long long *time_out = nullptr, *cpos = nullptr, *cneg = nullptr;
  double *density = nullptr, *current = nullptr, *field = nullptr;
  karl_status fail = KARL_OK;
};

}  // namespace

struct karl_server {
  int device = 0, num_sms = 0;
  karl_server_opts opts;
  ModelInfo model;
  std::vector<double> sigma;                   // channel-major host copy
  double* d_sig_t = nullptr;
  float* d_sigf = nullptr;
  double* d_cum = nullptr;                     // cumulative gas cross sections
  float* d_cumf = nullptr;
  unsigned char* d_mixed = nullptr;
  double* d_sig_cm = nullptr;
  // scattering-angle tables (NULL: every elastic channel isotropic)
  double* d_ang_pdf = nullptr;
  double* d_ang_cum = nullptr;
  float* d_ang_pdff = nullptr;
  float* d_ang_cumf = nullptr;
  // device control
  SlotDesc* d_desc = nullptr;
  SlotCtl* d_ctl = nullptr;
  MultiCtl* d_M = nullptr;
  int* d_cancel = nullptr;
  Ring ring;
  unsigned long long ring_cap = 0;
  char* d_arena = nullptr;
  Arena arena;
  // pinned host staging
  SlotDesc* h_desc = nullptr;
  SlotCtl* h_ctl = nullptr;
  unsigned* h_pubq = nullptr;
  unsigned long long* h_pubval = nullptr;
  int* h_done = nullptr;                       // mapped: written by the kernel
  int* h_state = nullptr;                      // pinned: slot states being published
  std::vector<unsigned> slot_gen;              // admissions into each slot so far (mod 2^24)
  int* d_done = nullptr;
  int* h_flag = nullptr;                       // pinned 1 (shutdown / cancel source)
  char* h_zero = nullptr;                      // pinned zeros: clears device memory by copy
  cudaStream_t kstream = nullptr, cstream = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;    // around the current launch
  bool running = false;
  unsigned long long seq = 0;                  // requests published so far
  std::vector<int> slot_req;                   // slot -> request index (-1 free)
  std::map<uint64_t, Request> reqs;
  std::deque<uint64_t> waiting;
  uint64_t next_id = 1;
  karl_server_stats stats;
  std::string err;
};

namespace {

karl_status sfail(karl_server* s, karl_status st, const char* fmt, ...) {
  char buf[2048];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (s) s->err = buf;
  return st;
}

#define SCK(call)                                                               \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess)                                                      \
      return sfail(srv, e_ == cudaErrorMemoryAllocation ? KARL_ENOMEM : KARL_ECUDA, "%s: %s", \
                   #call, cudaGetErrorString(e_));                              \
  } while (0)

// The persistent launch holds every SM, so nothing may launch a kernel while
// it runs (a memset is a kernel): device memory of a request is cleared by
// copies from pinned zeros, which the copy engines do beside the launch.
constexpr size_t ZERO_CHUNK = 16u << 20;

cudaError_t zero_by_copy(const karl_server* srv, void* dst, size_t bytes, cudaStream_t st) {
  char* d = (char*)dst;
  while (bytes) {
    const size_t n = std::min(bytes, ZERO_CHUNK);
    cudaError_t e = cudaMemcpyAsync(d, srv->h_zero, n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    d += n;
    bytes -= n;
  }
  return cudaSuccess;
}

size_t footprint(const Sizes& z) {
  size_t b = 0;
  b += 3 * up(z.n * 8) + up(z.n);                                   // primaries
  b += 2 * up(z.nz * 8) + 2 * up((z.nz + 1) * 8) + up((z.nq + 1) * 4);  // tables
  const size_t tallies = up(z.nspec * 8) + 2 * up(z.nt * 8) + 2 * up(z.cross_rg * 8) +
                         up(z.rec * 8) + up(LEDGER * 8) + up(MAXCH * 8);
  b += 2 * tallies;                                                 // both passes
  b += up(z.nch * z.nz * 8) + up(z.nch * (z.nz + 1) * 8) + up(z.nt * 8);  // fields, time1
  b += up(z.nt * 8) + 3 * up(z.cross * 8) + up((size_t)NSP * z.nz * z.ntb * 8) +
       up((size_t)NSP * z.nz * 8);                                   // outputs
  return b;
}

__global__ void k_ring_seq(unsigned long long* seq, unsigned long long cap) {
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < cap;
       i += (unsigned long long)gridDim.x * blockDim.x)
    seq[i] = i;
}

karl_status launch(karl_server* srv) {
  // reset the launch control (error words and the ring), keep the sequence counters
  MultiCtl zero;
  std::memset(&zero, 0, sizeof zero);
  SCK(cudaMemcpyAsync(&srv->d_M->c, &zero.c, sizeof(Control), cudaMemcpyHostToDevice,
                      srv->cstream));
  SCK(cudaMemsetAsync(srv->d_cancel, 0, sizeof(int), srv->cstream));
  // ring counters restart at 0, so every cell must be free at its position again
  k_ring_seq<<<1024, 256, 0, srv->cstream>>>(srv->ring.seq, srv->ring.cap);
  SCK(cudaGetLastError());
  SCK(cudaStreamSynchronize(srv->cstream));
  const bool f32 = srv->opts.precision == KARL_FP32;
  int bps = 0;
  SCK(multi_occupancy(f32, srv->opts.block_size, &bps));
  if (srv->opts.blocks_per_sm > 0) bps = std::min(bps, (int)srv->opts.blocks_per_sm);
  bps = std::max(bps, 1);
  TraceRange trace("karl server launch");
  SCK(cudaEventRecord(srv->ev0, srv->kstream));
  SCK(launch_multi(f32, srv->d_desc, srv->d_ctl, srv->d_M, srv->ring, srv->d_cancel,
                   (unsigned long long)(srv->opts.timeout_s * 1e9), srv->num_sms * bps,
                   srv->opts.block_size, srv->kstream));
  SCK(cudaEventRecord(srv->ev1, srv->kstream));
  srv->running = true;
  srv->stats.kernel_launches += 1;
  return KARL_OK;
}

// Put a request on the device and publish it to the (running) launch.
karl_status admit(karl_server* srv, Request& r) {
  Sizes z(r.g, r.z.size(), srv->model.nch, r.tabs.nq);
  int slot = -1;
  for (int i = 0; i < srv->opts.max_slots; ++i)
    if (srv->slot_req[i] < 0) { slot = i; break; }
  if (slot < 0) return KARL_EBUSY;
  size_t off = 0;
  if (!srv->arena.alloc(r.bytes, &off)) return KARL_EBUSY;
  r.slot = slot;
  r.off = off;
  char* p = srv->d_arena + off;
  auto take = [&](size_t bytes) {
    char* q = p;
    p += up(bytes);
    return q;
  };
  double* pz = (double*)take(z.n * 8);
  double* pe = (double*)take(z.n * 8);
  double* pmu = (double*)take(z.n * 8);
  uint8_t* psp = (uint8_t*)take(z.n);
  double* nseg = (double*)take(z.nz * 8);
  double* invn = (double*)take(z.nz * 8);
  double* col = (double*)take((z.nz + 1) * 8);
  double* faces = (double*)take((z.nz + 1) * 8);
  int* ginv = (int*)take((z.nq + 1) * 4);
  char* tally0 = p;
  struct PassBufs {
    unsigned long long *spec, *tpt, *trg, *xpos, *xneg, *rec, *led, *chan;
  } pb[2];
  for (int k = 0; k < 2; ++k) {
    pb[k].spec = (unsigned long long*)take(z.nspec * 8);
    pb[k].tpt = (unsigned long long*)take(z.nt * 8);
    pb[k].trg = (unsigned long long*)take(z.nt * 8);
    pb[k].xpos = (unsigned long long*)take(z.cross_rg * 8);
    pb[k].xneg = (unsigned long long*)take(z.cross_rg * 8);
    pb[k].rec = (unsigned long long*)take(z.rec * 8);
    pb[k].led = (unsigned long long*)take(LEDGER * 8);
    pb[k].chan = (unsigned long long*)take(MAXCH * 8);
  }
  const size_t tally_bytes = (size_t)(p - tally0);
  double* frate = (double*)take(z.nch * z.nz * 8);
  double* fcol = (double*)take(z.nch * (z.nz + 1) * 8);
  unsigned long long* time1 = (unsigned long long*)take(z.nt * 8);
  r.time_out = (unsigned long long*)take(z.nt * 8);
  r.cpos = (unsigned long long*)take(z.cross * 8);
  r.cneg = (unsigned long long*)take(z.cross * 8);
  r.current = (double*)take(z.cross * 8);
  r.field = (double*)take((size_t)NSP * z.nz * z.ntb * 8);
  r.density = (double*)take((size_t)NSP * z.nz * 8);
  if ((size_t)(p - (srv->d_arena + off)) > r.bytes) {
    srv->arena.release(off, r.bytes);
    return sfail(srv, KARL_ECUDA, "internal: request layout exceeds its footprint");
  }
  cudaStream_t cs = srv->cstream;
  if (z.n) {
    SCK(cudaMemcpyAsync(pz, r.z.data(), z.n * 8, cudaMemcpyHostToDevice, cs));
    SCK(cudaMemcpyAsync(pe, r.e.data(), z.n * 8, cudaMemcpyHostToDevice, cs));
    SCK(cudaMemcpyAsync(pmu, r.mu.data(), z.n * 8, cudaMemcpyHostToDevice, cs));
    SCK(cudaMemcpyAsync(psp, r.sp.data(), z.n, cudaMemcpyHostToDevice, cs));
  }
  SCK(cudaMemcpyAsync(nseg, r.nseg.data(), z.nz * 8, cudaMemcpyHostToDevice, cs));
  SCK(cudaMemcpyAsync(invn, r.tabs.invn.data(), z.nz * 8, cudaMemcpyHostToDevice, cs));
  SCK(cudaMemcpyAsync(col, r.tabs.col.data(), (z.nz + 1) * 8, cudaMemcpyHostToDevice, cs));
  SCK(cudaMemcpyAsync(faces, r.tabs.faces.data(), (z.nz + 1) * 8, cudaMemcpyHostToDevice, cs));
  SCK(cudaMemcpyAsync(ginv, r.tabs.ginv.data(), (z.nq + 1) * 4, cudaMemcpyHostToDevice, cs));
  SCK(zero_by_copy(srv, tally0, tally_bytes, cs));
  for (int c = 0; c < srv->model.nch; ++c)
    if (srv->model.kind[c] == CLUSTERING3) {
      SCK(cudaMemcpyAsync(frate + (size_t)c * z.nz, r.n2.data(), z.nz * 8,
                          cudaMemcpyHostToDevice, cs));
      SCK(cudaMemcpyAsync(fcol + (size_t)c * (z.nz + 1), r.col2.data(), (z.nz + 1) * 8,
                          cudaMemcpyHostToDevice, cs));
    }
  // descriptor
  const int final_pass = (r.n_passes == 2 && has_recombination(srv->model)) ? 2 : 1;
  SlotDesc& d = srv->h_desc[slot];
  std::memset(&d, 0, sizeof d);
  for (int k = 0; k < 2; ++k) {
    Params& P = d.P[k];
    fill_params(P, r.g, srv->model, k + 1, r.seed, r.tabs.nq, r.tabs.colmax);
    P.nseg = nseg;
    P.colgas = col;
    P.faces = faces;
    P.ginv = r.tabs.nq > 0 ? ginv : nullptr;
    P.sig = srv->d_sig_t;
    P.sigf = srv->d_sigf;
    P.invn = invn;
    P.cum = srv->d_cum;
    P.cumf = srv->d_cumf;
    P.mixed = srv->d_mixed;
    P.ang_pdf = srv->d_ang_pdf;
    P.ang_cum = srv->d_ang_cum;
    P.ang_pdff = srv->d_ang_pdff;
    P.ang_cumf = srv->d_ang_cumf;
    P.pid_offset = r.pid_offset;
    P.n_prim = (long long)z.n;
    P.pz = pz; P.pe = pe; P.pmu = pmu; P.psp = psp;
    P.spectrum = pb[k].spec;
    P.time_pt = pb[k].tpt;
    P.time_rg = pb[k].trg;
    P.xpos_rg = pb[k].xpos;
    P.xneg_rg = pb[k].xneg;
    P.recomb = pb[k].rec;
    P.ledger = pb[k].led;
    P.chan_count = pb[k].chan;
    P.per_primary = nullptr;
    for (int c = 0; c < srv->model.nch; ++c)
      if ((k == 1 && srv->model.kind[c] == RECOMBINATION) || srv->model.kind[c] == CLUSTERING3) {
        P.frate[c] = frate + (size_t)c * z.nz;
        P.fcol[c] = fcol + (size_t)c * (z.nz + 1);
      }
  }
  d.n_passes = final_pass;
  d.n_prim = (long long)z.n;
  d.time1 = time1;
  d.frate = frate;
  d.fcol = fcol;
  d.time_out = r.time_out;
  d.cpos_out = r.cpos;
  d.cneg_out = r.cneg;
  d.density = r.density;
  d.current = r.current;
  d.field = r.field;
  d.tsim = (double)r.n_decays / r.g.activity_bq;
  d.vol = (r.g.length_m / r.g.n_zbins) * r.g.area_m2;
  d.area = r.g.area_m2;
  d.sig_cm = srv->d_sig_cm;
  d.done_flag = srv->d_done + slot;
  const int fp = final_pass - 1;
  r.spec = pb[fp].spec;
  r.rec = pb[fp].rec;
  r.led = pb[fp].led;
  r.led1 = fp == 1 ? pb[0].led : nullptr;
  r.chan = pb[fp].chan;
  // A new generation for the slot.  Written in three ordered copies: the
  // control line with this generation's pass words and the state still empty,
  // then the descriptor, then the state "pass 1".  A lane that read the
  // previous request's state claims only on words of that generation, and a
  // lane that sees this descriptor also sees this generation's words.
  const unsigned gen = srv->slot_gen[slot] = (srv->slot_gen[slot] + 1) & 0xffffffu;
  SlotCtl& c = srv->h_ctl[slot];
  std::memset(&c, 0, sizeof c);
  c.word[0] = c.word[1] = (unsigned long long)(gen & 31u) << WORD_GEN_SHIFT;
  c.state = (int)(gen << 8) | SLOT_EMPTY;
  c.pass = 1;
  srv->h_done[slot] = 0;
  srv->h_state[slot] = (int)(gen << 8) | SLOT_PASS1;
  SCK(cudaMemcpyAsync(srv->d_ctl + slot, &c, sizeof c, cudaMemcpyHostToDevice, cs));
  SCK(cudaMemcpyAsync(srv->d_desc + slot, &d, sizeof d, cudaMemcpyHostToDevice, cs));
  SCK(cudaMemcpyAsync(&srv->d_ctl[slot].state, srv->h_state + slot, sizeof(int),
                      cudaMemcpyHostToDevice, cs));
  srv->slot_req[slot] = 1;
  if (z.n == 0) {
    // nothing to transport: zero outputs, finished at once
    const size_t out_bytes = (size_t)((char*)(r.density + (size_t)NSP * z.nz) - (char*)time1);
    SCK(zero_by_copy(srv, time1, out_bytes, cs));
    SCK(cudaStreamSynchronize(cs));
    srv->h_done[slot] = 1;
    r.state = REQ_ADMITTED;
    srv->stats.admitted += 1;
    return KARL_OK;
  }
  const unsigned long long q = srv->seq % MAX_SLOTS;
  srv->h_pubq[q] = (unsigned)slot;
  srv->h_pubval[q] = srv->seq + 1;
  SCK(cudaMemcpyAsync(srv->d_M->pubq + q, srv->h_pubq + q, sizeof(unsigned), cudaMemcpyHostToDevice,
                      cs));
  SCK(cudaMemcpyAsync(&srv->d_M->published, srv->h_pubval + q, sizeof(unsigned long long),
                      cudaMemcpyHostToDevice, cs));
  SCK(cudaStreamSynchronize(cs));
  srv->seq += 1;
  r.state = REQ_ADMITTED;
  srv->stats.admitted += 1;
  if (!srv->running) return launch(srv);
  return KARL_OK;
}

karl_status collect(karl_server* srv, Request& r) {
  Sizes z(r.g, r.z.size(), srv->model.nch, r.tabs.nq);
  cudaStream_t cs = srv->cstream;
  karl_tallies& o = r.out;
  SCK(cudaMemcpyAsync(o.spectrum, r.spec, z.nspec * 8, cudaMemcpyDeviceToHost, cs));
  SCK(cudaMemcpyAsync(o.time_fx, r.time_out, z.nt * 8, cudaMemcpyDeviceToHost, cs));
  SCK(cudaMemcpyAsync(o.cross_pos, r.cpos, z.cross * 8, cudaMemcpyDeviceToHost, cs));
  SCK(cudaMemcpyAsync(o.cross_neg, r.cneg, z.cross * 8, cudaMemcpyDeviceToHost, cs));
  SCK(cudaMemcpyAsync(o.recomb, r.rec, z.rec * 8, cudaMemcpyDeviceToHost, cs));
  SCK(cudaMemcpyAsync(o.ledger, r.led, LEDGER * 8, cudaMemcpyDeviceToHost, cs));
  unsigned long long led1[2] = {0, 0};
  if (r.led1)
    SCK(cudaMemcpyAsync(led1, r.led1 + L_N_COLL_ALL, sizeof led1, cudaMemcpyDeviceToHost, cs));
  if (o.chan_count && srv->model.nch)
    SCK(cudaMemcpyAsync(o.chan_count, r.chan, (size_t)srv->model.nch * 8, cudaMemcpyDeviceToHost,
                        cs));
  if (o.density)
    SCK(cudaMemcpyAsync(o.density, r.density, (size_t)NSP * z.nz * 8, cudaMemcpyDeviceToHost, cs));
  if (o.current)
    SCK(cudaMemcpyAsync(o.current, r.current, z.cross * 8, cudaMemcpyDeviceToHost, cs));
  if (o.field)
    SCK(cudaMemcpyAsync(o.field, r.field, (size_t)NSP * z.nz * z.ntb * 8, cudaMemcpyDeviceToHost,
                        cs));
  SCK(cudaStreamSynchronize(cs));
  if (r.z.empty()) {
    std::memset(o.spectrum, 0, z.nspec * 8);
    std::memset(o.recomb, 0, z.rec * 8);
    std::memset(o.ledger, 0, LEDGER * 8);
    if (o.chan_count && srv->model.nch) std::memset(o.chan_count, 0, (size_t)srv->model.nch * 8);
  }
  // the ledger is the last pass's; its all-pass counts take pass 1's as well
  ((int64_t*)o.ledger)[L_N_COLL_ALL] += (int64_t)led1[0];
  ((int64_t*)o.ledger)[L_N_FLIGHT_ALL] += (int64_t)led1[1];
  srv->stats.collisions += ((int64_t*)o.ledger)[L_N_COLL_ALL];
  srv->arena.release(r.off, r.bytes);
  srv->slot_req[r.slot] = -1;
  r.state = REQ_FINISHED;
  srv->stats.completed += 1;
  return KARL_OK;
}

void free_request_memory(Request& r) {
  std::vector<double>().swap(r.z);
  std::vector<double>().swap(r.e);
  std::vector<double>().swap(r.mu);
  std::vector<uint8_t>().swap(r.sp);
}

// the launch has stopped: read its error, fail what it left unfinished
karl_status reap_launch(karl_server* srv) {
  if (!srv->running) return KARL_OK;
  cudaError_t q = cudaStreamQuery(srv->kstream);
  if (q == cudaErrorNotReady) return KARL_OK;
  srv->running = false;
  if (q != cudaSuccess) return sfail(srv, KARL_ECUDA, "launch: %s", cudaGetErrorString(q));
  Control hc;
  SCK(cudaMemcpy(&hc, &srv->d_M->c, sizeof hc, cudaMemcpyDeviceToHost));
  float ms = 0.0f;
  if (cudaEventElapsedTime(&ms, srv->ev0, srv->ev1) == cudaSuccess) srv->stats.kernel_ms += ms;
  srv->stats.lane_occupancy =
      hc.busy_iters + hc.idle_iters
          ? (double)hc.busy_lane_iters / (32.0 * (double)(hc.busy_iters + hc.idle_iters))
          : 0.0;
  if (hc.error == ERR_CAPACITY) {
    // products overflowed the shared ring: grow it for the next launch
    // (at most 2^26 cells: a request's live count has 28 bits in its pass word)
    if (srv->ring_cap < (1ULL << 26)) srv->ring_cap *= 4;
  }
  if (hc.error != 0) {
    const karl_status st = hc.error == ERR_TIMEOUT ? KARL_ETIMEOUT
                         : hc.error == ERR_CANCELLED ? KARL_ECANCELLED : KARL_ECAPACITY;
    // what the stopped launch left unfinished, for the error message
    std::string detail;
    {
      MultiCtl hm;
      std::vector<SlotCtl> hs(MAX_SLOTS);
      if (cudaMemcpy(&hm, srv->d_M, sizeof hm, cudaMemcpyDeviceToHost) == cudaSuccess &&
          cudaMemcpy(hs.data(), srv->d_ctl, sizeof(SlotCtl) * MAX_SLOTS,
                     cudaMemcpyDeviceToHost) == cudaSuccess) {
        char b[256];
        snprintf(b, sizeof b, "; published %llu adopted %llu done %llu ring head %llu tail %llu",
                 hm.published, hm.adopted, hm.done_count, hm.c.head, hm.c.tail);
        detail += b;
        for (auto& kv : srv->reqs) {
          const Request& r = kv.second;
          if (r.state != REQ_ADMITTED || srv->h_done[r.slot]) continue;
          const SlotCtl& c = hs[r.slot];
          snprintf(b, sizeof b, "; slot %d state %d gen %u pass %d claimed/live %lld/%llu %lld/%llu of %zu",
                   r.slot, state_kind(c.state), state_gen(c.state), c.pass, word_next(c.word[0]),
                   word_live(c.word[0]), word_next(c.word[1]), word_live(c.word[1]), r.z.size());
          detail += b;
        }
      }
    }
    for (auto& kv : srv->reqs) {
      Request& r = kv.second;
      if (r.state == REQ_ADMITTED && !srv->h_done[r.slot]) {
        r.state = REQ_FAILED;
        r.fail = st;
        srv->arena.release(r.off, r.bytes);
        srv->slot_req[r.slot] = -1;
      }
    }
    // a fresh start for what comes next: slots free, ring and counters reset
    SCK(cudaMemset(srv->d_ctl, 0, sizeof(SlotCtl) * MAX_SLOTS));
    SCK(cudaMemset(srv->d_M, 0, sizeof(MultiCtl)));
    srv->seq = 0;
    if (hc.error == ERR_CAPACITY) {
      // (re)allocate a larger ring
      return sfail(srv, KARL_ECAPACITY, "particle ring overflow; grown for later requests");
    }
    return sfail(srv, st, "launch stopped (error %d)%s", hc.error, detail.c_str());
  }
  return KARL_OK;
}

karl_status ensure_ring(karl_server* srv) {
  if (srv->ring.z && srv->ring.cap == srv->ring_cap) return KARL_OK;
  Ring& R = srv->ring;
  if (R.z) {
    cudaFree(R.z); cudaFree(R.eq); cudaFree(R.mu); cudaFree(R.node); cudaFree(R.tal);
    cudaFree(R.pid); cudaFree(R.ev); cudaFree(R.sj); cudaFree(R.seq);
  }
  std::memset(&R, 0, sizeof R);
  const size_t n = (size_t)srv->ring_cap;
  SCK(cudaMalloc(&R.z, n * 8));
  SCK(cudaMalloc(&R.eq, n * 8));
  SCK(cudaMalloc(&R.mu, n * 8));
  SCK(cudaMalloc(&R.node, n * 8));
  SCK(cudaMalloc(&R.tal, n * 8));
  SCK(cudaMalloc(&R.pid, n * 8));
  SCK(cudaMalloc(&R.ev, n * 4));
  SCK(cudaMalloc(&R.sj, n * 4));
  SCK(cudaMalloc(&R.seq, n * 8));
  R.cap = srv->ring_cap;
  R.mask = srv->ring_cap - 1;
  k_ring_seq<<<1024, 256, 0, srv->cstream>>>(R.seq, R.cap);
  SCK(cudaGetLastError());
  SCK(cudaStreamSynchronize(srv->cstream));
  return KARL_OK;
}

// collect finished requests, then admit waiting ones in arrival order
karl_status progress(karl_server* srv) {
  karl_status st = reap_launch(srv);
  if (st && st != KARL_ECAPACITY) return st;
  for (auto& kv : srv->reqs) {
    Request& r = kv.second;
    if (r.state == REQ_ADMITTED && srv->h_done[r.slot]) {
      karl_status c = collect(srv, r);
      if (c) return c;
      free_request_memory(r);
    }
  }
  if (!srv->running) {
    karl_status rs = ensure_ring(srv);
    if (rs) return rs;
  }
  while (!srv->waiting.empty()) {
    Request& r = srv->reqs[srv->waiting.front()];
    karl_status a = admit(srv, r);
    if (a == KARL_EBUSY) break;
    if (a) return a;
    srv->waiting.pop_front();
  }
  if (!srv->running) {
    // published work whose launch has already left (it saw shutdown before
    // the request was published): start another launch for it
    for (auto& kv : srv->reqs)
      if (kv.second.state == REQ_ADMITTED && !srv->h_done[kv.second.slot]) {
        karl_status l = launch(srv);
        if (l) return l;
        break;
      }
  }
  srv->stats.waiting = (int64_t)srv->waiting.size();
  srv->stats.arena_bytes_in_use = (int64_t)srv->arena.in_use;
  srv->stats.arena_bytes_peak = (int64_t)srv->arena.peak;
  return KARL_OK;
}

karl_status set_shutdown(karl_server* srv, int v) {
  *srv->h_flag = v;
  SCK(cudaMemcpyAsync(&srv->d_M->shutdown, srv->h_flag, sizeof(int), cudaMemcpyHostToDevice,
                      srv->cstream));
  SCK(cudaStreamSynchronize(srv->cstream));
  return KARL_OK;
}

}  // namespace

extern "C" {

karl_status karl_server_create(const karl_xs* xs, const karl_server_opts* opts,
                               karl_server** out) {
  if (!out) return KARL_EINVAL;
  *out = nullptr;
  if (!xs_ok(xs)) return KARL_EINVAL;
  karl_server_opts o;
  std::memset(&o, 0, sizeof o);
  if (opts) o = *opts;
  if (o.precision != KARL_FP64 && o.precision != KARL_FP32) return KARL_EINVAL;
  if (o.max_slots == 0) o.max_slots = 256;
  if (o.max_slots < 1 || o.max_slots > MAX_SLOTS) return KARL_EINVAL;
  if (o.hbm_budget_bytes == 0) o.hbm_budget_bytes = 16LL << 30;
  if (o.hbm_budget_bytes < (1LL << 20)) return KARL_EINVAL;
  if (!(o.timeout_s > 0)) o.timeout_s = 3600.0;
  if (o.block_size == 0) o.block_size = 256;
  if (o.block_size < 32 || o.block_size > 256 || o.block_size % 32) return KARL_EINVAL;
  karl_server* srv = new (std::nothrow) karl_server();
  if (!srv) return KARL_ENOMEM;
  std::memset(&srv->stats, 0, sizeof srv->stats);
  std::memset(&srv->ring, 0, sizeof srv->ring);
  srv->opts = o;
  srv->model = model_info(xs);
  srv->slot_req.assign(MAX_SLOTS, -1);
  srv->ring_cap = 1ULL << 22;
  auto bail = [&](karl_status s) {
    karl_server_destroy(srv);
    return s;
  };
  if (cudaGetDevice(&srv->device) ||
      cudaDeviceGetAttribute(&srv->num_sms, cudaDevAttrMultiProcessorCount, srv->device))
    return bail(KARL_ECUDA);
  std::vector<double> sig_t, cum;
  std::vector<float> sigf, cumf;
  std::vector<unsigned char> mixed;
  node_major_tables(xs, sig_t, sigf);
  gas_cum_tables(xs, srv->model, cum, cumf, mixed);
  const size_t nsig = std::max<size_t>(sig_t.size(), 1);
  const size_t ncum = std::max<size_t>(cum.size(), 2);
  if (cudaMalloc(&srv->d_cum, ncum * 8) || cudaMalloc(&srv->d_cumf, ncum * 4) ||
      cudaMalloc(&srv->d_mixed, mixed.size()))
    return bail(KARL_ENOMEM);
  if (cudaMemcpy(srv->d_mixed, mixed.data(), mixed.size(), cudaMemcpyHostToDevice) ||
      (!cum.empty() &&
       (cudaMemcpy(srv->d_cum, cum.data(), cum.size() * 8, cudaMemcpyHostToDevice) ||
        cudaMemcpy(srv->d_cumf, cumf.data(), cumf.size() * 4, cudaMemcpyHostToDevice))))
    return bail(KARL_ECUDA);
  srv->sigma.assign(xs->sigma_m2, xs->sigma_m2 + (size_t)xs->n_channels * xs->n_energy);
  if (cudaMalloc(&srv->d_sig_t, nsig * 8) || cudaMalloc(&srv->d_sigf, nsig * 4) ||
      cudaMalloc(&srv->d_sig_cm, nsig * 8) ||
      cudaMalloc(&srv->d_desc, sizeof(SlotDesc) * MAX_SLOTS) ||
      cudaMalloc(&srv->d_ctl, sizeof(SlotCtl) * MAX_SLOTS) ||
      cudaMalloc(&srv->d_M, sizeof(MultiCtl)) || cudaMalloc(&srv->d_cancel, sizeof(int)) ||
      cudaMalloc(&srv->d_arena, (size_t)o.hbm_budget_bytes))
    return bail(KARL_ENOMEM);
  if (cudaHostAlloc(&srv->h_desc, sizeof(SlotDesc) * MAX_SLOTS, cudaHostAllocDefault) ||
      cudaHostAlloc(&srv->h_ctl, sizeof(SlotCtl) * MAX_SLOTS, cudaHostAllocDefault) ||
      cudaHostAlloc(&srv->h_pubq, sizeof(unsigned) * MAX_SLOTS, cudaHostAllocDefault) ||
      cudaHostAlloc(&srv->h_pubval, sizeof(unsigned long long) * MAX_SLOTS, cudaHostAllocDefault) ||
      cudaHostAlloc(&srv->h_done, sizeof(int) * MAX_SLOTS, cudaHostAllocMapped) ||
      cudaHostAlloc(&srv->h_state, sizeof(int) * MAX_SLOTS, cudaHostAllocDefault) ||
      cudaHostGetDevicePointer(&srv->d_done, srv->h_done, 0) ||
      cudaHostAlloc(&srv->h_flag, sizeof(int), cudaHostAllocDefault) ||
      cudaHostAlloc(&srv->h_zero, ZERO_CHUNK, cudaHostAllocDefault))
    return bail(KARL_ENOMEM);
  std::memset(srv->h_zero, 0, ZERO_CHUNK);
  std::memset(srv->h_done, 0, sizeof(int) * MAX_SLOTS);
  srv->slot_gen.assign(MAX_SLOTS, 0);
  srv->arena.init((size_t)o.hbm_budget_bytes);
  if (sig_t.size() &&
      (cudaMemcpy(srv->d_sig_t, sig_t.data(), sig_t.size() * 8, cudaMemcpyHostToDevice) ||
       cudaMemcpy(srv->d_sigf, sigf.data(), sigf.size() * 4, cudaMemcpyHostToDevice) ||
       cudaMemcpy(srv->d_sig_cm, srv->sigma.data(), srv->sigma.size() * 8,
                  cudaMemcpyHostToDevice)))
    return bail(KARL_ECUDA);
  {
    std::vector<double> apdf, acum;
    std::vector<float> apdff, acumf;
    try {
      angular_tables(xs, apdf, acum, apdff, acumf);
    } catch (...) {
      return bail(KARL_ENOMEM);
    }
    if (!apdf.empty()) {
      const size_t na = apdf.size();
      if (cudaMalloc(&srv->d_ang_pdf, na * 8) || cudaMalloc(&srv->d_ang_cum, na * 8) ||
          cudaMalloc(&srv->d_ang_pdff, na * 4) || cudaMalloc(&srv->d_ang_cumf, na * 4))
        return bail(KARL_ENOMEM);
      if (cudaMemcpy(srv->d_ang_pdf, apdf.data(), na * 8, cudaMemcpyHostToDevice) ||
          cudaMemcpy(srv->d_ang_cum, acum.data(), na * 8, cudaMemcpyHostToDevice) ||
          cudaMemcpy(srv->d_ang_pdff, apdff.data(), na * 4, cudaMemcpyHostToDevice) ||
          cudaMemcpy(srv->d_ang_cumf, acumf.data(), na * 4, cudaMemcpyHostToDevice))
        return bail(KARL_ECUDA);
    }
  }
  if (cudaMemset(srv->d_ctl, 0, sizeof(SlotCtl) * MAX_SLOTS) ||
      cudaMemset(srv->d_M, 0, sizeof(MultiCtl)) || cudaMemset(srv->d_cancel, 0, sizeof(int)) ||
      cudaStreamCreateWithFlags(&srv->kstream, cudaStreamNonBlocking) ||
      cudaStreamCreateWithFlags(&srv->cstream, cudaStreamNonBlocking) ||
      cudaEventCreate(&srv->ev0) || cudaEventCreate(&srv->ev1))
    return bail(KARL_ECUDA);
  if (ensure_ring(srv)) return bail(KARL_ENOMEM);
  *out = srv;
  return KARL_OK;
}

karl_status karl_server_layout(const karl_server* srv, const karl_geometry* g, karl_layout* out) {
  if (!srv || !out || !geometry_ok(g)) return KARL_EINVAL;
  Sizes z(*g, 0, srv->model.nch, 0);
  out->spectrum = (int64_t)z.nspec;
  out->time_fx = (int64_t)z.nt;
  out->cross = (int64_t)z.cross;
  out->recomb = (int64_t)z.rec;
  out->ledger = LEDGER;
  out->chan_count = srv->model.nch;
  out->density = (int64_t)NSP * z.nz;
  out->current = (int64_t)z.cross;
  out->field = (int64_t)NSP * z.nz * z.ntb;
  return KARL_OK;
}

karl_status karl_server_submit(karl_server* srv, const karl_geometry* g, const karl_primaries* pr,
                               uint64_t seed, int32_t n_passes, karl_tallies* out,
                               uint64_t* req_id) {
  if (!srv) return KARL_EINVAL;
  srv->err.clear();
  if (!geometry_ok(g)) return sfail(srv, KARL_EINVAL, "invalid geometry");
  if (!pr || pr->n < 0 || pr->on_device) return sfail(srv, KARL_EINVAL, "primaries: host arrays");
  if (pr->n > MAX_REQUEST_PRIMARIES)
    return sfail(srv, KARL_EINVAL, "a request holds at most 2^31 - 1 primaries");
  if (pr->n > 0 && (!pr->z_m || !pr->e_ev || !pr->mu || !pr->species))
    return sfail(srv, KARL_EINVAL, "primaries: NULL array");
  if (!(pr->n_decays > 0)) return sfail(srv, KARL_EINVAL, "n_decays must be > 0");
  if (n_passes != 1 && n_passes != 2) return sfail(srv, KARL_EINVAL, "n_passes must be 1 or 2");
  if (!out || out->on_device || !out->spectrum || !out->time_fx || !out->cross_pos ||
      !out->cross_neg || !out->recomb || !out->ledger || (srv->model.nch && !out->chan_count))
    return sfail(srv, KARL_EINVAL, "tally buffers: host arrays required");
  if (!req_id) return sfail(srv, KARL_EINVAL, "req_id is NULL");
  for (int64_t i = 0; i < pr->n; ++i) {
    const double zi = pr->z_m[i], ei = pr->e_ev[i], mi = pr->mu[i];
    if (!(zi >= 0.0 && zi <= g->length_m) || !(ei > 0.0 && ei < 1e12) ||
        !(mi >= -1.0 && mi <= 1.0) || pr->species[i] >= NSP)
      return sfail(srv, KARL_EINVAL, "primary %lld out of range", (long long)i);
  }
  Request r;
  try {
    r.nseg.assign(g->n_seg_m3, g->n_seg_m3 + g->n_zbins);
    r.z.assign(pr->z_m, pr->z_m + pr->n);
    r.e.assign(pr->e_ev, pr->e_ev + pr->n);
    r.mu.assign(pr->mu, pr->mu + pr->n);
    r.sp.assign(pr->species, pr->species + pr->n);
    bool three_body = false;
    for (int c = 0; c < srv->model.nch; ++c) three_body |= srv->model.kind[c] == CLUSTERING3;
    if (three_body) square_column(r.nseg.data(), g->n_zbins, g->length_m, r.n2, r.col2);
  } catch (...) {
    return sfail(srv, KARL_ENOMEM, "host copy of the request");
  }
  r.g = *g;
  r.g.n_seg_m3 = nullptr;
  r.tabs = column_tables(r.nseg.data(), g->n_zbins, g->length_m);
  r.n_decays = pr->n_decays;
  r.pid_offset = pr->pid_offset;
  r.seed = seed;
  r.n_passes = n_passes;
  r.out = *out;
  Sizes z(*g, (size_t)pr->n, srv->model.nch, r.tabs.nq);
  r.bytes = footprint(z);
  if (r.bytes > srv->arena.size)
    return sfail(srv, KARL_EINVAL, "request footprint %zu B exceeds the budget", r.bytes);
  r.id = srv->next_id++;
  *req_id = r.id;
  srv->reqs.emplace(r.id, std::move(r));
  srv->waiting.push_back(*req_id);
  srv->stats.submitted += 1;
  return progress(srv);
}

karl_status karl_server_poll(karl_server* srv, uint64_t req_id, int* done) {
  if (!srv || !done) return KARL_EINVAL;
  *done = 0;
  auto it = srv->reqs.find(req_id);
  if (it == srv->reqs.end()) return sfail(srv, KARL_ENOTFOUND, "unknown request %llu",
                                          (unsigned long long)req_id);
  karl_status st = progress(srv);
  it = srv->reqs.find(req_id);
  if (it->second.state == REQ_FAILED) {
    const karl_status f = it->second.fail;
    srv->reqs.erase(it);
    return f;
  }
  if (it->second.state == REQ_FINISHED) {
    *done = 1;
    srv->stats.collected += 1;
    srv->reqs.erase(it);
    return KARL_OK;
  }
  return st == KARL_ECAPACITY ? KARL_OK : st;
}

karl_status karl_server_run_all(karl_server* srv) {
  if (!srv) return KARL_EINVAL;
  // everything that fits goes on the device before the launch starts
  karl_status st = progress(srv);
  if (st && st != KARL_ECAPACITY) return st;
  st = set_shutdown(srv, 1);
  if (st) return st;
  for (;;) {
    st = progress(srv);
    if (st && st != KARL_ECAPACITY) return st;
    bool open = false;
    for (auto& kv : srv->reqs)
      if (kv.second.state == REQ_QUEUED || kv.second.state == REQ_ADMITTED) open = true;
    if (!open) break;
    if (!srv->running) {
      // published work with no launch (e.g. admitted after the last one left)
      bool pending = false;
      for (auto& kv : srv->reqs)
        if (kv.second.state == REQ_ADMITTED && !srv->h_done[kv.second.slot]) pending = true;
      if (pending) {
        st = launch(srv);
        if (st) return st;
      }
    }
    struct timespec ts = {0, 200000};
    nanosleep(&ts, nullptr);
  }
  if (srv->running) {
    cudaStreamSynchronize(srv->kstream);
    st = reap_launch(srv);
    if (st && st != KARL_ECAPACITY) return st;
  }
  return set_shutdown(srv, 0);
}

karl_status karl_server_get_stats(const karl_server* srv, karl_server_stats* out) {
  if (!srv || !out) return KARL_EINVAL;
  *out = srv->stats;
  return KARL_OK;
}

const char* karl_server_last_error(const karl_server* srv) { return srv ? srv->err.c_str() : ""; }

void karl_server_destroy(karl_server* srv) {
  if (!srv) return;
  if (srv->running && srv->d_M && srv->h_flag) {
    *srv->h_flag = 1;
    cudaMemcpyAsync(&srv->d_M->shutdown, srv->h_flag, sizeof(int), cudaMemcpyHostToDevice,
                    srv->cstream);
    cudaStreamSynchronize(srv->cstream);
    cudaStreamSynchronize(srv->kstream);
  }
  Ring& R = srv->ring;
  if (R.z) {
    cudaFree(R.z); cudaFree(R.eq); cudaFree(R.mu); cudaFree(R.node); cudaFree(R.tal);
    cudaFree(R.pid); cudaFree(R.ev); cudaFree(R.sj); cudaFree(R.seq);
  }
  cudaFree(srv->d_sig_t); cudaFree(srv->d_sigf); cudaFree(srv->d_sig_cm);
  cudaFree(srv->d_cum); cudaFree(srv->d_cumf); cudaFree(srv->d_mixed);
  cudaFree(srv->d_ang_pdf); cudaFree(srv->d_ang_cum); cudaFree(srv->d_ang_pdff);
  cudaFree(srv->d_ang_cumf);
  cudaFree(srv->d_desc); cudaFree(srv->d_ctl); cudaFree(srv->d_M); cudaFree(srv->d_cancel);
  cudaFree(srv->d_arena);
  if (srv->h_desc) cudaFreeHost(srv->h_desc);
  if (srv->h_ctl) cudaFreeHost(srv->h_ctl);
  if (srv->h_pubq) cudaFreeHost(srv->h_pubq);
  if (srv->h_pubval) cudaFreeHost(srv->h_pubval);
  if (srv->h_done) cudaFreeHost(srv->h_done);
  if (srv->h_state) cudaFreeHost(srv->h_state);
  if (srv->h_flag) cudaFreeHost(srv->h_flag);
  if (srv->h_zero) cudaFreeHost(srv->h_zero);
  if (srv->ev0) cudaEventDestroy(srv->ev0);
  if (srv->ev1) cudaEventDestroy(srv->ev1);
  if (srv->kstream) cudaStreamDestroy(srv->kstream);
  if (srv->cstream) cudaStreamDestroy(srv->cstream);
  delete srv;
}

}  // extern "C"
