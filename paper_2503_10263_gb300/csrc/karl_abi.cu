// karl_abi.cu - C ABI of the KARL transport path (declared in include/karl.h).
//
// Host orchestration only: argument checks, device tables, the pass sequence
// (pass 1 without recombination, target fields, pass 2), queue regrowth, and
// small kernels for the prefix sums of the range-add tallies and the
// normalisation of Eq. target_field_density and the current of Sec. 2.3.
// Every step of the transport itself runs in transport.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/karl.h"
#include "host_common.h"
#include "orbit.cuh"

namespace karl {
cudaError_t launch_transport(bool f32, const Params& P, const Ring& R, Control* ctl,
                             const volatile int* cancel, unsigned long long timeout_ns, int grid,
                             int block, cudaStream_t st);
cudaError_t transport_occupancy(bool f32, const Params& P, int block, int* blocks_per_sm);
cudaError_t transport_setup();
cudaError_t launch_orbit(const Params& P, const OrbitDev& O, int grid, int block,
                         cudaStream_t st);
cudaError_t orbit_occupancy(int block, int* blocks_per_sm);
}  // namespace karl

using namespace karl;

namespace {

const double Q_TIME = 1125899906842624.0;
const double C_LIGHT = 299792458.0;

// Device memory of contexts comes from a library-wide memory pool per device,
// allocated and freed in stream order on a library stream.  A plain cudaFree
// waits for every kernel on the device -- also for a served session's
// persistent launch, which runs until its session closes, so a context freed
// meanwhile (by a destructor, from any thread) would stall both.  Pool frees
// wait for nothing, and the pool keeps freed memory for later contexts.
struct DevicePools {
  std::mutex m;
  cudaMemPool_t pool[64] = {};
  cudaStream_t stream[64] = {};
};
DevicePools& device_pools() {
  static DevicePools d;
  return d;
}

// The pool and the allocation stream of the current device (created once).
cudaError_t current_pool(cudaMemPool_t* pool, cudaStream_t* st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  DevicePools& d = device_pools();
  std::lock_guard<std::mutex> lk(d.m);
  if (!d.pool[dev]) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    e = cudaMemPoolCreate(&p, &props);
    if (e != cudaSuccess) return e;
    unsigned long long keep = ~0ULL;                 // never hand freed memory back
    e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    cudaStream_t s = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(p);
      return e;
    }
    d.pool[dev] = p;
    d.stream[dev] = s;
  }
  *pool = d.pool[dev];
  *st = d.stream[dev];
  return cudaSuccess;
}

// Buffers replaced by a larger one while a call runs may still be read by work
// that call queued; they are kept as `retired` and freed at the start of the
// context's next call (every call returns only after its work is done).
template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t st = nullptr;                         // allocation stream of p's device
  std::vector<T*> retired;
  cudaError_t ensure(size_t count) {
    if (count <= n && p) return cudaSuccess;
    if (p) retired.push_back(p);
    p = nullptr;
    n = 0;
    cudaMemPool_t pool;
    cudaError_t e = current_pool(&pool, &st);
    if (e != cudaSuccess) return e;
    void* q = nullptr;
    e = cudaMallocFromPoolAsync(&q, std::max<size_t>(count, 1) * sizeof(T), pool, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // usable from every stream
    if (e == cudaSuccess) {
      p = (T*)q;
      n = std::max<size_t>(count, 1);
    }
    return e;
  }
  void drop_retired() {
    for (T* q : retired) cudaFreeAsync(q, st);
    retired.clear();
  }
  void release() {
    drop_retired();
    if (p) cudaFreeAsync(p, st);
    p = nullptr;
    n = 0;
  }
};

const int zero_word = 0;

// A page-locked word holding 1: the source of the copy that cancels a run.
const int* pinned_one() {
  static int* one = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    if (cudaHostAlloc((void**)&one, sizeof(int), cudaHostAllocDefault) == cudaSuccess) *one = 1;
    else one = nullptr;
  });
  return one;
}

}  // namespace

struct karl_ctx {
  int device = 0;
  int num_sms = 0;
  karl_geometry geom;          // copy (n_seg_m3 points at nseg below)
  ModelInfo model;
  cudaStream_t own_stream = nullptr;
  // copies of the inputs
  double L = 0, dz = 0, area = 1, activity = 1, e_cut = 0, max_life = 0, kT = 0;
  unsigned max_coll = 0;
  int nz = 0, ntb = 1, nspec = 1;
  double spec_bin = 1;
  double mass[NSP] = {};
  double target_mass = 1;
  int n_energy = 0, nch = 0;
  double e_min = 1, e_max = 2;
  double eps_ion = 8;
  std::vector<double> nseg, sigma;
  std::vector<int> kind, sin, sout;
  std::vector<double> loss;
  // device tables
  DevBuf<double> d_nseg, d_colgas, d_faces, d_sig, d_sig_t, d_frate, d_fcol, d_time1;
  DevBuf<double> d_invn, d_cum;              // 1/n per segment; cumulative gas cross sections
  DevBuf<float> d_cumf;
  DevBuf<unsigned char> d_mixed;
  DevBuf<int> d_ginv;
  int nq = 0;
  double colmax = 0;
  DevBuf<float> d_sigf;
  DevBuf<double> d_ang_pdf, d_ang_cum;       // scattering-angle tables (empty: isotropic)
  DevBuf<double> d_n2, d_col2;               // n^2 and its column (three-body clustering)
  DevBuf<float> d_ang_pdff, d_ang_cumf;
  cudaStream_t cancel_stream = nullptr;
  // device work buffers
  DevBuf<double> d_pz, d_pe, d_pmu;
  DevBuf<uint8_t> d_psp;
  DevBuf<unsigned long long> d_spec, d_tpt, d_trg, d_xpos, d_xneg, d_recomb, d_ledger, d_chan,
      d_pp, d_time, d_cpos, d_cneg;
  DevBuf<double> d_density, d_current, d_field;
  DevBuf<int> d_bad;
  // ring
  DevBuf<double> r_z, r_mu, r_tal;
  DevBuf<long long> r_eq;
  DevBuf<unsigned long long> r_node, r_pid, r_seq;
  DevBuf<unsigned> r_ev, r_sj;
  unsigned long long ring_cap = 0;
  DevBuf<Control> d_ctlbuf;
  DevBuf<int> d_cancelbuf;
  // sums over the cycles of a continuous-update run
  DevBuf<unsigned long long> c_spec, c_time, c_cpos, c_cneg, c_rec, c_led, c_chan, c_pp, d_recin;
  // full-orbit runs: primaries, the lists of two generations, raw tallies
  DevBuf<double> o_px, o_py, o_pz, o_pe, o_pmu, o_pphi, o_ez, o_energy, o_end, o_u2edge,
      o_edge2;
  DevBuf<uint8_t> o_psp, o_lsp[2];
  DevBuf<double> o_lx[2], o_ly[2], o_lz[2], o_lux[2], o_luy[2], o_luz[2];
  DevBuf<unsigned long long> o_lnode[2], o_lpid[2];
  DevBuf<unsigned long long> o_tz, o_tr, o_xp, o_xn, o_ro, o_ri, o_wall, o_spec, o_led, o_chan,
      o_pp, o_cnt;
  DevBuf<int> o_err;
  Control* d_ctl = nullptr;     // = d_ctlbuf.p
  int* d_cancel = nullptr;      // = d_cancelbuf.p, device word polled by the kernel
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  karl_run_stats stats;
  std::string err;
  // every device buffer of the context
  template <class F>
  void each_buf(F f) {
    f(d_nseg); f(d_colgas); f(d_faces); f(d_sig); f(d_sig_t); f(d_frate); f(d_fcol); f(d_time1);
    f(d_invn); f(d_cum); f(d_cumf); f(d_mixed);
    f(d_ginv); f(d_sigf); f(d_ang_pdf); f(d_ang_cum); f(d_ang_pdff); f(d_ang_cumf); f(d_n2);
    f(d_col2); f(d_pz); f(d_pe); f(d_pmu); f(d_psp); f(d_spec); f(d_tpt); f(d_trg); f(d_xpos);
    f(d_xneg); f(d_recomb); f(d_ledger); f(d_chan); f(d_pp); f(d_time); f(d_cpos); f(d_cneg);
    f(d_density); f(d_current); f(d_field); f(d_bad); f(r_z); f(r_mu); f(r_tal); f(r_eq);
    f(r_node); f(r_pid); f(r_seq); f(r_ev); f(r_sj); f(d_ctlbuf); f(d_cancelbuf);
    f(c_spec); f(c_time); f(c_cpos); f(c_cneg); f(c_rec); f(c_led); f(c_chan); f(c_pp); f(d_recin);
    f(o_px); f(o_py); f(o_pz); f(o_pe); f(o_pmu); f(o_pphi); f(o_ez); f(o_energy); f(o_end);
    f(o_u2edge); f(o_edge2);
    f(o_psp); f(o_tz); f(o_tr); f(o_xp); f(o_xn); f(o_ro); f(o_ri); f(o_wall); f(o_spec);
    f(o_led); f(o_chan); f(o_pp); f(o_cnt); f(o_err);
    for (int g = 0; g < 2; ++g) {
      f(o_lsp[g]); f(o_lx[g]); f(o_ly[g]); f(o_lz[g]); f(o_lux[g]); f(o_luy[g]); f(o_luz[g]);
      f(o_lnode[g]); f(o_lpid[g]);
    }
  }
  // buffers replaced during earlier calls (none of their work is in flight now)
  void drop_retired() {
    each_buf([](auto& b) { b.drop_retired(); });
  }
};

namespace {

karl_status fail(karl_ctx* c, karl_status s, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return s;
}

karl_status cuda_fail(karl_ctx* c, cudaError_t e, const char* where) {
  karl_status s = (e == cudaErrorMemoryAllocation) ? KARL_ENOMEM : KARL_ECUDA;
  return fail(c, s, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);  \
  } while (0)

// ---------------------------------------------------------------------------
// small kernels

__global__ void k_ring_init(unsigned long long* seq, unsigned long long cap) {
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < cap;
       i += (unsigned long long)gridDim.x * blockDim.x)
    seq[i] = i;
}

__global__ void k_check_primaries(const double* z, const double* e, const double* mu,
                                  const uint8_t* sp, long long n, double L, int* bad) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    bool ok = z[i] >= 0.0 && z[i] <= L && e[i] > 0.0 && e[i] < 1e12 && mu[i] >= -1.0 &&
              mu[i] <= 1.0 && sp[i] < NSP;
    if (!ok) atomicAdd(bad, 1);
  }
}

// time = point adds + prefix of range adds, per (species, energy bin)
__global__ void k_finalize_time(const unsigned long long* pt, const unsigned long long* rg,
                                unsigned long long* out, int nz, int ntb) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NSP * ntb) return;
  int s = t / ntb, b = t % ntb;
  unsigned long long acc = 0;
  for (int row = 0; row < nz + 2; ++row) {
    size_t i = ((size_t)s * (nz + 2) + row) * ntb + b;
    acc += rg[i];
    out[i] = pt[i] + acc;
  }
}

__global__ void k_finalize_cross(const unsigned long long* rg, unsigned long long* out, int nz) {
  int s = threadIdx.x;
  if (s >= NSP) return;
  unsigned long long acc = 0;
  for (int k = 0; k <= nz; ++k) {
    acc += rg[(size_t)s * (nz + 2) + k];
    out[(size_t)s * (nz + 1) + k] = acc;
  }
}

__device__ double sigma_interp(const double* sig, int n, double e_min, double e_max, double loss,
                               double e) {
  if (!(e > loss)) return 0.0;
  double h = log(e_max / e_min) / (double)(n - 1);
  double x = log(e / e_min) / h;
  int i = (int)floor(x);
  double f;
  if (i < 0) { i = 0; f = 0.0; }
  else if (i > n - 2) { i = n - 2; f = 1.0; }
  else f = x - (double)i;
  return (1.0 - f) * sig[i] + f * sig[i + 1];
}

struct FieldArgs {
  int nz, ntb, n_energy, nch;
  double tsim, vol, dz, e_min, e_max, me;
  int kind[MAXCH], sin[MAXCH], sout[MAXCH];
  double loss[MAXCH];
};

// Target fields from summed time tallies (Eq. target_field_density with t_sim
// of Eq. simulated_time) and, for the cycles of the continuous update, the
// deletions logged in the partner's field (its -N/V term: a bin's density
// takes the segment's deletions in proportion to its time; below zero it
// counts as zero).  recomb NULL: no deletions (pass 2 of a two-pass run).
// Electron impactor: ion density.  Ion impactor: sum over electron energy
// bins of n_e(E_b) sigma(E_b) v(E_b).
__global__ void k_build_fields(FieldArgs A, const unsigned long long* time1,
                               const unsigned long long* recomb, const double* sig, double* frate,
                               double* fcol) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= A.nch * A.nz) return;
  int k = t / A.nz, j = t % A.nz;
  if (A.kind[k] != RECOMBINATION) return;
  int partner = A.sout[k];
  const unsigned long long* tj = time1 + ((size_t)partner * (A.nz + 2) + (j + 1)) * A.ntb;
  double ttot = 0.0, del = 0.0;
  if (recomb) {
    for (int b = 0; b < A.ntb; ++b) ttot += (double)tj[b];
    del = (double)recomb[(size_t)partner * A.nz + j] / A.vol;
  }
  double acc = 0.0;
  for (int b = 0; b < A.ntb; ++b) {
    double n = (double)tj[b] / Q_TIME / (A.tsim * A.vol);
    if (recomb && ttot > 0.0) n -= del * ((double)tj[b] / ttot);
    if (A.sin[k] == SP_E) {
      acc += n;
    } else {
      double eb = A.e_min * pow(A.e_max / A.e_min, (b + 0.5) / A.ntb);
      double x = eb / A.me;
      double v = C_LIGHT * sqrt(x * (2.0 + x)) / (1.0 + x);
      acc += fmax(n, 0.0) * sigma_interp(sig + (size_t)k * A.n_energy, A.n_energy, A.e_min,
                                         A.e_max, A.loss[k], eb) * v;
    }
  }
  frate[(size_t)k * A.nz + j] = fmax(acc, 0.0);
}

__global__ void k_field_columns(const double* frate, double* fcol, int nch, int nz, double dz) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nch) return;
  double c = 0.0;
  fcol[(size_t)k * (nz + 1)] = 0.0;
  for (int j = 0; j < nz; ++j) {
    c += frate[(size_t)k * nz + j] * dz;
    fcol[(size_t)k * (nz + 1) + j + 1] = c;
  }
}

// field_del: the field output takes its deletions as the cycles' fields do
__global__ void k_normalize(const unsigned long long* time, const unsigned long long* time1,
                            const unsigned long long* recomb, const unsigned long long* cpos,
                            const unsigned long long* cneg, double* density, double* current,
                            double* field, int nz, int ntb, double tsim, double vol, double area,
                            int field_del) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < NSP * nz) {
    int s = t / nz, j = t % nz;
    double tsum = 0.0, t1tot = 0.0;
    if (field_del)
      for (int b = 0; b < ntb; ++b) t1tot += (double)time1[((size_t)s * (nz + 2) + (j + 1)) * ntb + b];
    const double del = field_del ? (double)recomb[(size_t)s * nz + j] / vol : 0.0;
    for (int b = 0; b < ntb; ++b) {
      size_t idx = ((size_t)s * (nz + 2) + (j + 1)) * ntb + b;
      tsum += (double)time[idx] / Q_TIME;
      if (field) {
        double nb = (double)time1[idx] / Q_TIME / (tsim * vol);
        if (field_del && t1tot > 0.0) nb -= del * ((double)time1[idx] / t1tot);
        field[((size_t)s * nz + j) * ntb + b] = field_del ? fmax(nb, 0.0) : nb;
      }
    }
    if (density) density[(size_t)s * nz + j] =
        tsum / (tsim * vol) - (double)recomb[(size_t)s * nz + j] / vol;
  }
  if (t < NSP * (nz + 1) && current) {
    current[t] = ((double)cpos[t] - (double)cneg[t]) / (area * tsim);
  }
}

__global__ void k_accumulate(unsigned long long* dst, const unsigned long long* src, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    dst[i] += src[i];
}

int grid_for(size_t n, int block) {
  size_t g = (n + block - 1) / block;
  return (int)std::min<size_t>(std::max<size_t>(g, 1), 4096);
}

// ---------------------------------------------------------------------------
// helpers

karl_status stage_primaries(karl_ctx* ctx, const karl_primaries* pr, cudaStream_t st,
                            const double** z, const double** e, const double** mu,
                            const uint8_t** sp) {
  if (pr->n == 0) {
    *z = *e = *mu = nullptr;
    *sp = nullptr;
    return KARL_OK;
  }
  if (!pr->z_m || !pr->e_ev || !pr->mu || !pr->species)
    return fail(ctx, KARL_EINVAL, "primaries: NULL array");
  size_t n = (size_t)pr->n;
  if (pr->on_device) {
    *z = pr->z_m; *e = pr->e_ev; *mu = pr->mu; *sp = pr->species;
  } else {
    for (size_t i = 0; i < n; ++i) {
      double zi = pr->z_m[i], ei = pr->e_ev[i], mi = pr->mu[i];
      if (!(zi >= 0.0 && zi <= ctx->L) || !(ei > 0.0 && ei < 1e12) || !(mi >= -1.0 && mi <= 1.0) ||
          pr->species[i] >= NSP)
        return fail(ctx, KARL_EINVAL, "primary %zu out of range (z=%g e=%g mu=%g species=%d)", i,
                    zi, ei, mi, (int)pr->species[i]);
    }
    CK(ctx->d_pz.ensure(n));
    CK(ctx->d_pe.ensure(n));
    CK(ctx->d_pmu.ensure(n));
    CK(ctx->d_psp.ensure(n));
    CK(cudaMemcpyAsync(ctx->d_pz.p, pr->z_m, n * 8, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ctx->d_pe.p, pr->e_ev, n * 8, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ctx->d_pmu.p, pr->mu, n * 8, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ctx->d_psp.p, pr->species, n, cudaMemcpyHostToDevice, st));
    *z = ctx->d_pz.p; *e = ctx->d_pe.p; *mu = ctx->d_pmu.p; *sp = ctx->d_psp.p;
    return KARL_OK;
  }
  // device primaries: check on the device
  CK(ctx->d_bad.ensure(1));
  CK(cudaMemsetAsync(ctx->d_bad.p, 0, sizeof(int), st));
  k_check_primaries<<<grid_for(n, 256), 256, 0, st>>>(*z, *e, *mu, *sp, (long long)n, ctx->L,
                                                      ctx->d_bad.p);
  CK(cudaGetLastError());
  ctx->stats.kernel_launches += 1;
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, ctx->d_bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (bad) return fail(ctx, KARL_EINVAL, "%d primaries out of range", bad);
  return KARL_OK;
}

size_t n_time(const karl_ctx* c) { return (size_t)NSP * (c->nz + 2) * c->ntb; }
size_t n_spec(const karl_ctx* c) { return (size_t)2 * NSP * (c->nspec + 1); }
size_t n_cross_rg(const karl_ctx* c) { return (size_t)NSP * (c->nz + 2); }
size_t n_cross(const karl_ctx* c) { return (size_t)NSP * (c->nz + 1); }
size_t n_recomb(const karl_ctx* c) { return (size_t)NSP * c->nz; }

// Default threads per block of the transport kernel (resident blocks per SM:
// the occupancy maximum): one block of 512 threads per SM.  With at most 128
// registers a thread that keeps as many warps resident as two blocks of 256,
// and the single block's share of shared memory also holds the pass-2 field
// tables.  Measured on the config-2 step (5e6 decays) against 256 x 2:
// FP64 2.881e9 against 2.872e9 collisions/s, FP32 5.44e9 against 5.26e9.
int default_block(bool) { return 512; }

karl_status ensure_ring(karl_ctx* ctx, unsigned long long cap) {
  if (ctx->ring_cap >= cap) return KARL_OK;
  size_t n = (size_t)cap;
  CK(ctx->r_z.ensure(n));
  CK(ctx->r_mu.ensure(n));
  CK(ctx->r_tal.ensure(n));
  CK(ctx->r_eq.ensure(n));
  CK(ctx->r_node.ensure(n));
  CK(ctx->r_pid.ensure(n));
  CK(ctx->r_seq.ensure(n));
  CK(ctx->r_ev.ensure(n));
  CK(ctx->r_sj.ensure(n));
  ctx->ring_cap = cap;
  return KARL_OK;
}

// Kernel parameters of one pass of this context (device buffers set by the caller).
void base_params(const karl_ctx* c, Params& P, const karl_run_opts* o, int pass) {
  fill_params(P, c->geom, c->model, pass, o->seed, c->nq, c->colmax);
  P.nseg = c->d_nseg.p;
  P.colgas = c->d_colgas.p;
  P.faces = c->d_faces.p;
  P.ginv = c->nq > 0 ? c->d_ginv.p : nullptr;
  P.sig = c->d_sig_t.p;
  P.sigf = c->d_sigf.p;
  P.invn = c->d_invn.p;
  P.cum = c->d_cum.p;
  P.cumf = c->d_cumf.p;
  P.mixed = c->d_mixed.p;
  for (int k = 0; k < c->nch; ++k)
    if (c->kind[k] == CLUSTERING3) {
      P.frate[k] = c->d_n2.p;
      P.fcol[k] = c->d_col2.p;
    }
  if (c->model.ang_sets > 0) {
    P.ang_pdf = c->d_ang_pdf.p;
    P.ang_cum = c->d_ang_cum.p;
    P.ang_pdff = c->d_ang_pdff.p;
    P.ang_cumf = c->d_ang_cumf.p;
  }
}

// One pass into the context's raw tally buffers (which are zeroed first).
karl_status run_one_pass(karl_ctx* ctx, const karl_primaries* pr, const karl_run_opts* o,
                         int pass, const double* pz, const double* pe, const double* pmu,
                         const uint8_t* psp, bool per_primary, cudaStream_t st) {
  TraceRange trace(pass == 1 ? "karl transport pass 1" : "karl transport pass 2");
  size_t nt = n_time(ctx);
  CK(ctx->d_spec.ensure(n_spec(ctx)));
  CK(ctx->d_tpt.ensure(nt));
  CK(ctx->d_trg.ensure(nt));
  CK(ctx->d_xpos.ensure(n_cross_rg(ctx)));
  CK(ctx->d_xneg.ensure(n_cross_rg(ctx)));
  CK(ctx->d_recomb.ensure(n_recomb(ctx)));
  CK(ctx->d_ledger.ensure(LEDGER));
  CK(ctx->d_chan.ensure(MAXCH));
  if (per_primary) CK(ctx->d_pp.ensure((size_t)std::max<int64_t>(pr->n, 1)));
  bool f32 = o->precision == KARL_FP32;
  int block = o->block_size > 0 ? o->block_size : default_block(f32);
  int grid = 0;
  // The shared product ring: a power of two of cells, at least 2^22 and
  // about one cell per primary up to 2^24 (1 GiB), so that in a large pass the
  // spilled products rarely fill it to the level at which lanes stop taking
  // new primaries; it grows (the pass rerun) only if it overflows.
  unsigned long long want = 1ULL << 22;
  while (want < (unsigned long long)pr->n && want < (1ULL << 24)) want <<= 1;
  unsigned long long cap = ctx->ring_cap > want ? ctx->ring_cap : want;
  double timeout = o->timeout_s > 0 ? o->timeout_s : 600.0;
  for (int attempt = 0; attempt < 4; ++attempt) {
    karl_status rs = ensure_ring(ctx, cap);
    if (rs != KARL_OK) return rs;
    CK(cudaMemsetAsync(ctx->d_spec.p, 0, n_spec(ctx) * 8, st));
    CK(cudaMemsetAsync(ctx->d_tpt.p, 0, nt * 8, st));
    CK(cudaMemsetAsync(ctx->d_trg.p, 0, nt * 8, st));
    CK(cudaMemsetAsync(ctx->d_xpos.p, 0, n_cross_rg(ctx) * 8, st));
    CK(cudaMemsetAsync(ctx->d_xneg.p, 0, n_cross_rg(ctx) * 8, st));
    CK(cudaMemsetAsync(ctx->d_recomb.p, 0, n_recomb(ctx) * 8, st));
    CK(cudaMemsetAsync(ctx->d_ledger.p, 0, LEDGER * 8, st));
    CK(cudaMemsetAsync(ctx->d_chan.p, 0, MAXCH * 8, st));
    if (per_primary) CK(cudaMemsetAsync(ctx->d_pp.p, 0, (size_t)std::max<int64_t>(pr->n, 1) * 8, st));
    CK(cudaMemsetAsync(ctx->d_ctl, 0, sizeof(Control), st));
    k_ring_init<<<grid_for((size_t)ctx->ring_cap, 256), 256, 0, st>>>(ctx->r_seq.p, ctx->ring_cap);
    CK(cudaGetLastError());
    ctx->stats.kernel_launches += 1;

    Params P;
    base_params(ctx, P, o, pass);
    if (pass == 2) {
      for (int k = 0; k < ctx->nch; ++k) {
        if (ctx->kind[k] != RECOMBINATION) continue;
        P.frate[k] = ctx->d_frate.p + (size_t)k * ctx->nz;
        P.fcol[k] = ctx->d_fcol.p + (size_t)k * (ctx->nz + 1);
      }
    }
    P.pid_offset = pr->pid_offset;
    P.n_prim = pr->n;
    P.pz = pz; P.pe = pe; P.pmu = pmu; P.psp = psp;
    P.spectrum = ctx->d_spec.p;
    P.time_pt = ctx->d_tpt.p;
    P.time_rg = ctx->d_trg.p;
    P.xpos_rg = ctx->d_xpos.p;
    P.xneg_rg = ctx->d_xneg.p;
    P.recomb = ctx->d_recomb.p;
    P.ledger = ctx->d_ledger.p;
    P.chan_count = ctx->d_chan.p;
    P.per_primary = per_primary ? ctx->d_pp.p : nullptr;
    if (grid == 0) {
      int bps = 0;
      CK(transport_occupancy(f32, P, block, &bps));
      if (o->blocks_per_sm > 0) bps = std::min(bps, (int)o->blocks_per_sm);
      if (bps < 1) bps = 1;
      grid = ctx->num_sms * bps;
    }

    Ring R;
    R.z = ctx->r_z.p; R.eq = ctx->r_eq.p; R.mu = ctx->r_mu.p; R.node = ctx->r_node.p;
    R.tal = ctx->r_tal.p; R.pid = ctx->r_pid.p; R.ev = ctx->r_ev.p; R.sj = ctx->r_sj.p;
    R.seq = ctx->r_seq.p; R.cap = ctx->ring_cap; R.mask = ctx->ring_cap - 1;

    CK(cudaMemsetAsync(ctx->d_cancel, 0, sizeof(int), st));
    CK(cudaEventRecord(ctx->ev0, st));
    CK(launch_transport(f32, P, R, ctx->d_ctl, ctx->d_cancel,
                        (unsigned long long)(timeout * 1e9), grid, block, st));
    CK(cudaEventRecord(ctx->ev1, st));
    Control hc;
    CK(cudaMemcpyAsync(&hc, ctx->d_ctl, sizeof hc, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    float ms = 0;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    int pi = pass - 1;
    ctx->stats.kernel_ms[pi] = ms;
    ctx->stats.particles[pi] = (int64_t)hc.particles;
    ctx->stats.spilled[pi] = (int64_t)hc.spilled;
    ctx->stats.idle_warp_frac[pi] =
        hc.busy_iters + hc.idle_iters
            ? (double)hc.idle_iters / (double)(hc.busy_iters + hc.idle_iters)
            : 0.0;
    ctx->stats.tail_ms[pi] =
        hc.t_end > hc.t_claimed && hc.t_claimed ? (double)(hc.t_end - hc.t_claimed) * 1e-6 : 0.0;
    ctx->stats.lane_occupancy[pi] =
        hc.busy_iters + hc.idle_iters
            ? (double)hc.busy_lane_iters / (32.0 * (double)(hc.busy_iters + hc.idle_iters))
            : 0.0;
    ctx->stats.grid_blocks = grid;
    ctx->stats.block_size = block;
    ctx->stats.queue_capacity = (int32_t)std::min<unsigned long long>(ctx->ring_cap, 0x7fffffff);
    ctx->stats.kernel_launches += 1;
    if (hc.error == ERR_CAPACITY) {       // ring too small: grow and rerun the pass
      cap = ctx->ring_cap * 4;
      continue;
    }
    if (hc.error == ERR_TIMEOUT) return fail(ctx, KARL_ETIMEOUT, "transport kernel timed out");
    if (hc.error == ERR_CANCELLED) return fail(ctx, KARL_ECANCELLED, "run cancelled");
    if (hc.error != 0) return fail(ctx, KARL_ECUDA, "transport kernel error %d", hc.error);
    long long led[LEDGER];
    CK(cudaMemcpy(led, ctx->d_ledger.p, sizeof led, cudaMemcpyDeviceToHost));
    ctx->stats.collisions[pi] = led[L_N_COLL];
    ctx->stats.flights[pi] = led[L_N_FLIGHT];
    // finalize range adds
    CK(ctx->d_time.ensure(nt));
    CK(ctx->d_cpos.ensure(n_cross(ctx)));
    CK(ctx->d_cneg.ensure(n_cross(ctx)));
    k_finalize_time<<<grid_for((size_t)NSP * ctx->ntb, 64), 64, 0, st>>>(
        ctx->d_tpt.p, ctx->d_trg.p, ctx->d_time.p, ctx->nz, ctx->ntb);
    k_finalize_cross<<<1, 32, 0, st>>>(ctx->d_xpos.p, ctx->d_cpos.p, ctx->nz);
    k_finalize_cross<<<1, 32, 0, st>>>(ctx->d_xneg.p, ctx->d_cneg.p, ctx->nz);
    CK(cudaGetLastError());
    ctx->stats.kernel_launches += 3;
    return KARL_OK;
  }
  return fail(ctx, KARL_ECAPACITY, "particle ring overflow at capacity %llu",
              (unsigned long long)ctx->ring_cap);
}

karl_status build_fields(karl_ctx* ctx, const unsigned long long* d_time1,
                         const unsigned long long* d_recomb, double n_decays, cudaStream_t st) {
  TraceRange trace("karl target fields");
  FieldArgs A;
  std::memset(&A, 0, sizeof A);
  A.nz = ctx->nz;
  A.ntb = ctx->ntb;
  A.n_energy = ctx->n_energy;
  A.nch = ctx->nch;
  A.tsim = n_decays / ctx->activity;
  A.vol = ctx->dz * ctx->area;
  A.dz = ctx->dz;
  A.e_min = ctx->e_min;
  A.e_max = ctx->e_max;
  A.me = ctx->mass[SP_E];
  for (int k = 0; k < ctx->nch; ++k) {
    A.kind[k] = ctx->kind[k];
    A.sin[k] = ctx->sin[k];
    A.sout[k] = ctx->sout[k];
    A.loss[k] = ctx->loss[k];
  }
  size_t nk = (size_t)std::max(ctx->nch, 1);
  CK(ctx->d_frate.ensure(nk * ctx->nz));
  CK(ctx->d_fcol.ensure(nk * (ctx->nz + 1)));
  CK(cudaMemsetAsync(ctx->d_frate.p, 0, nk * ctx->nz * 8, st));
  k_build_fields<<<grid_for((size_t)ctx->nch * ctx->nz, 256), 256, 0, st>>>(
      A, d_time1, d_recomb, ctx->d_sig.p, ctx->d_frate.p, ctx->d_fcol.p);
  k_field_columns<<<1, 32, 0, st>>>(ctx->d_frate.p, ctx->d_fcol.p, ctx->nch, ctx->nz, ctx->dz);
  CK(cudaGetLastError());
  ctx->stats.kernel_launches += 2;
  return KARL_OK;
}

karl_status copy_out(karl_ctx* ctx, void* dst, const void* src, size_t bytes, bool dst_dev,
                     cudaStream_t st) {
  if (!dst || bytes == 0) return KARL_OK;
  CK(cudaMemcpyAsync(dst, src, bytes, dst_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     st));
  return KARL_OK;
}

karl_status check_opts(karl_ctx* ctx, const karl_run_opts* o) {
  if (!o) return fail(ctx, KARL_EINVAL, "opts is NULL");
  if (o->precision != KARL_FP64 && o->precision != KARL_FP32)
    return fail(ctx, KARL_EINVAL, "precision must be KARL_FP64 or KARL_FP32");
  if (o->block_size != 0 && (o->block_size < 32 || o->block_size > 512 || o->block_size % 32))
    return fail(ctx, KARL_EINVAL, "block_size must be a multiple of 32 in [32, 512]");
  return KARL_OK;
}

}  // namespace

// ===========================================================================
// C ABI

extern "C" {

const char* karl_status_string(karl_status s) {
  switch (s) {
    case KARL_OK: return "ok";
    case KARL_EINVAL: return "invalid argument";
    case KARL_ENOMEM: return "out of memory";
    case KARL_ECUDA: return "CUDA error";
    case KARL_ETIMEOUT: return "timed out";
    case KARL_EOVERFLOW: return "tally overflow";
    case KARL_ECAPACITY: return "particle queue capacity exceeded";
    case KARL_ECANCELLED: return "cancelled";
    case KARL_EBUSY: return "busy";
    case KARL_ENOTFOUND: return "not found";
  }
  return "unknown status";
}

const char* karl_last_error(const karl_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

karl_status karl_create(const karl_geometry* g, const karl_xs* x, karl_ctx** out) {
  if (!out) return KARL_EINVAL;
  *out = nullptr;
  if (!geometry_ok(g) || !xs_ok(x)) return KARL_EINVAL;
  karl_ctx* ctx = new (std::nothrow) karl_ctx();
  if (!ctx) return KARL_ENOMEM;
  std::memset(&ctx->stats, 0, sizeof ctx->stats);
  auto bail = [&](karl_status s) {
    karl_destroy(ctx);
    return s;
  };
  if (cudaGetDevice(&ctx->device) != cudaSuccess) return bail(KARL_ECUDA);
  if (cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device) !=
      cudaSuccess)
    return bail(KARL_ECUDA);
  ctx->L = g->length_m;
  ctx->nz = g->n_zbins;
  ctx->dz = g->length_m / g->n_zbins;
  ctx->area = g->area_m2;
  ctx->activity = g->activity_bq;
  ctx->e_cut = g->e_cut_ev;
  ctx->max_coll = g->max_collisions;
  ctx->max_life = g->max_lifetime_s;
  ctx->kT = HOST_KB_EV * g->gas_temperature_k;
  ctx->ntb = g->n_tebins;
  ctx->nspec = g->n_spec_bins;
  ctx->spec_bin = g->spec_bin_ev;
  for (int s = 0; s < NSP; ++s) ctx->mass[s] = g->species_mass_ev[s];
  ctx->target_mass = g->target_mass_ev;
  ctx->n_energy = x->n_energy;
  ctx->e_min = x->e_min_ev;
  ctx->e_max = x->e_max_ev;
  ctx->nch = x->n_channels;
  ctx->eps_ion = x->ioniz_eps_ev;
  try {
    ctx->nseg.assign(g->n_seg_m3, g->n_seg_m3 + g->n_zbins);
    for (int k = 0; k < x->n_channels; ++k) {
      ctx->kind.push_back(x->kind[k]);
      ctx->sin.push_back(x->species_in[k]);
      ctx->sout.push_back(x->species_out[k]);
      ctx->loss.push_back(x->loss_ev[k]);
    }
    ctx->sigma.assign(x->sigma_m2, x->sigma_m2 + (size_t)x->n_channels * x->n_energy);
  } catch (...) {
    return bail(KARL_ENOMEM);
  }
  ctx->geom = *g;
  ctx->geom.n_seg_m3 = ctx->nseg.data();
  ctx->model = model_info(x);
  const ColumnTables tabs = column_tables(ctx->nseg.data(), ctx->nz, ctx->L);
  ctx->nq = tabs.nq;
  ctx->colmax = tabs.colmax;
  std::vector<double> sig_t, cum;
  std::vector<float> sigf, cumf;
  std::vector<unsigned char> mixed;
  try {
    node_major_tables(x, sig_t, sigf);
    gas_cum_tables(x, ctx->model, cum, cumf, mixed);
  } catch (...) {
    return bail(KARL_ENOMEM);
  }
  size_t nsig = std::max<size_t>(ctx->sigma.size(), 1);
  size_t nsig2 = std::max<size_t>(sig_t.size(), 1);
  const size_t ncum = std::max<size_t>(cum.size(), 2);
  if (ctx->d_invn.ensure(ctx->nz) || ctx->d_cum.ensure(ncum) || ctx->d_cumf.ensure(ncum) ||
      ctx->d_mixed.ensure(mixed.size()) ||
      cudaMemcpy(ctx->d_invn.p, tabs.invn.data(), ctx->nz * 8, cudaMemcpyHostToDevice) ||
      cudaMemcpy(ctx->d_mixed.p, mixed.data(), mixed.size(), cudaMemcpyHostToDevice) ||
      (!cum.empty() &&
       (cudaMemcpy(ctx->d_cum.p, cum.data(), cum.size() * 8, cudaMemcpyHostToDevice) ||
        cudaMemcpy(ctx->d_cumf.p, cumf.data(), cumf.size() * 4, cudaMemcpyHostToDevice))))
    return bail(KARL_ENOMEM);
  if (ctx->d_nseg.ensure(ctx->nz) || ctx->d_colgas.ensure(ctx->nz + 1) ||
      ctx->d_faces.ensure(ctx->nz + 1) ||
      ctx->d_sig.ensure(nsig) || ctx->d_sig_t.ensure(nsig2) || ctx->d_sigf.ensure(nsig2) ||
      ctx->d_ledger.ensure(LEDGER) || ctx->d_ginv.ensure(ctx->nq + 1))
    return bail(KARL_ENOMEM);
  if (cudaMemcpy(ctx->d_nseg.p, ctx->nseg.data(), ctx->nz * 8, cudaMemcpyHostToDevice) ||
      cudaMemcpy(ctx->d_colgas.p, tabs.col.data(), (ctx->nz + 1) * 8, cudaMemcpyHostToDevice) ||
      cudaMemcpy(ctx->d_faces.p, tabs.faces.data(), (ctx->nz + 1) * 8, cudaMemcpyHostToDevice) ||
      cudaMemcpy(ctx->d_ginv.p, tabs.ginv.data(), (ctx->nq + 1) * sizeof(int),
                 cudaMemcpyHostToDevice) ||
      (ctx->sigma.size() &&
       (cudaMemcpy(ctx->d_sig.p, ctx->sigma.data(), ctx->sigma.size() * 8, cudaMemcpyHostToDevice) ||
        cudaMemcpy(ctx->d_sig_t.p, sig_t.data(), sig_t.size() * 8, cudaMemcpyHostToDevice) ||
        cudaMemcpy(ctx->d_sigf.p, sigf.data(), sigf.size() * 4, cudaMemcpyHostToDevice))))
    return bail(KARL_ECUDA);
  if (has_kind(x, CLUSTERING3)) {
    std::vector<double> n2, col2;
    try {
      square_column(ctx->nseg.data(), ctx->nz, ctx->L, n2, col2);
    } catch (...) {
      return bail(KARL_ENOMEM);
    }
    if (ctx->d_n2.ensure(ctx->nz) || ctx->d_col2.ensure(ctx->nz + 1)) return bail(KARL_ENOMEM);
    if (cudaMemcpy(ctx->d_n2.p, n2.data(), ctx->nz * 8, cudaMemcpyHostToDevice) ||
        cudaMemcpy(ctx->d_col2.p, col2.data(), (ctx->nz + 1) * 8, cudaMemcpyHostToDevice))
      return bail(KARL_ECUDA);
  }
  {
    std::vector<double> apdf, acum;
    std::vector<float> apdff, acumf;
    try {
      angular_tables(x, apdf, acum, apdff, acumf);
    } catch (...) {
      return bail(KARL_ENOMEM);
    }
    if (!apdf.empty()) {
      const size_t na = apdf.size();
      if (ctx->d_ang_pdf.ensure(na) || ctx->d_ang_cum.ensure(na) || ctx->d_ang_pdff.ensure(na) ||
          ctx->d_ang_cumf.ensure(na))
        return bail(KARL_ENOMEM);
      if (cudaMemcpy(ctx->d_ang_pdf.p, apdf.data(), na * 8, cudaMemcpyHostToDevice) ||
          cudaMemcpy(ctx->d_ang_cum.p, acum.data(), na * 8, cudaMemcpyHostToDevice) ||
          cudaMemcpy(ctx->d_ang_pdff.p, apdff.data(), na * 4, cudaMemcpyHostToDevice) ||
          cudaMemcpy(ctx->d_ang_cumf.p, acumf.data(), na * 4, cudaMemcpyHostToDevice))
        return bail(KARL_ECUDA);
    }
  }
  if (transport_setup() != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking) ||
      cudaStreamCreateWithFlags(&ctx->cancel_stream, cudaStreamNonBlocking) ||
      ctx->d_ctlbuf.ensure(1) || ctx->d_cancelbuf.ensure(1) || !pinned_one() ||
      cudaMemcpy(ctx->d_cancelbuf.p, &zero_word, sizeof(int), cudaMemcpyHostToDevice) ||
      cudaEventCreate(&ctx->ev0) || cudaEventCreate(&ctx->ev1))
    return bail(KARL_ECUDA);
  ctx->d_ctl = ctx->d_ctlbuf.p;
  ctx->d_cancel = ctx->d_cancelbuf.p;
  *out = ctx;
  return KARL_OK;
}

void karl_cancel(karl_ctx* ctx) {
  // a copy on a stream of its own runs while the transport kernel is running
  if (ctx && ctx->d_cancel && ctx->cancel_stream) {
    cudaMemcpyAsync(ctx->d_cancel, pinned_one(), sizeof(int), cudaMemcpyHostToDevice,
                    ctx->cancel_stream);
    cudaStreamSynchronize(ctx->cancel_stream);
  }
}

karl_status karl_tally_layout(const karl_ctx* c, karl_layout* o) {
  if (!c || !o) return KARL_EINVAL;
  o->spectrum = (int64_t)n_spec(c);
  o->time_fx = (int64_t)n_time(c);
  o->cross = (int64_t)n_cross(c);
  o->recomb = (int64_t)n_recomb(c);
  o->ledger = LEDGER;
  o->chan_count = c->nch;
  o->density = (int64_t)NSP * c->nz;
  o->current = (int64_t)n_cross(c);
  o->field = (int64_t)NSP * c->nz * c->ntb;
  return KARL_OK;
}

karl_status karl_last_stats(const karl_ctx* c, karl_run_stats* o) {
  if (!c || !o) return KARL_EINVAL;
  *o = c->stats;
  return KARL_OK;
}

karl_status karl_run_pass(karl_ctx* ctx, const karl_primaries* pr, const karl_run_opts* o,
                          int32_t pass, const uint64_t* field_time_in, karl_tallies* out) {
  if (!ctx) return KARL_EINVAL;
  ctx->err.clear();
  ctx->drop_retired();
  if (!pr || !out || pr->n < 0) return fail(ctx, KARL_EINVAL, "NULL argument or n < 0");
  karl_status s = check_opts(ctx, o);
  if (s) return s;
  if (pass != 1 && pass != 2) return fail(ctx, KARL_EINVAL, "pass must be 1 or 2");
  if (pass == 2 && !field_time_in) return fail(ctx, KARL_EINVAL, "pass 2 needs field_time_in");
  if (pass == 2 && !(pr->n_decays > 0)) return fail(ctx, KARL_EINVAL, "n_decays must be > 0");
  if (!out->spectrum || !out->time_fx || !out->cross_pos || !out->cross_neg || !out->recomb ||
      !out->ledger || (ctx->nch > 0 && !out->chan_count))
    return fail(ctx, KARL_EINVAL, "tally buffer is NULL");
  cudaStream_t st = o->stream ? (cudaStream_t)o->stream : ctx->own_stream;
  const double *pz, *pe, *pmu;
  const uint8_t* psp;
  ctx->stats.kernel_launches = 0;
  s = stage_primaries(ctx, pr, st, &pz, &pe, &pmu, &psp);
  if (s) return s;
  if (pass == 2) {
    CK(ctx->d_time1.ensure(n_time(ctx)));
    CK(cudaMemcpyAsync(ctx->d_time1.p, field_time_in, n_time(ctx) * 8, cudaMemcpyHostToDevice, st));
    s = build_fields(ctx, (const unsigned long long*)ctx->d_time1.p, nullptr,
                     (double)pr->n_decays, st);
    if (s) return s;
  }
  bool pp = out->per_primary != nullptr && pr->n > 0;
  s = run_one_pass(ctx, pr, o, pass, pz, pe, pmu, psp, pp, st);
  if (s) return s;
  // add raw tallies into the caller's buffers
  struct Item { void* dst; const void* src; size_t n; };
  Item items[] = {
      {out->spectrum, ctx->d_spec.p, n_spec(ctx)}, {out->time_fx, ctx->d_time.p, n_time(ctx)},
      {out->cross_pos, ctx->d_cpos.p, n_cross(ctx)}, {out->cross_neg, ctx->d_cneg.p, n_cross(ctx)},
      {out->recomb, ctx->d_recomb.p, n_recomb(ctx)}, {out->ledger, ctx->d_ledger.p, (size_t)LEDGER},
      {out->chan_count, ctx->d_chan.p, (size_t)ctx->nch},
      {pp ? out->per_primary : nullptr, ctx->d_pp.p, (size_t)pr->n}};
  for (const Item& it : items) {
    if (!it.dst || it.n == 0) continue;
    if (out->on_device) {
      k_accumulate<<<grid_for(it.n, 256), 256, 0, st>>>((unsigned long long*)it.dst,
                                                         (const unsigned long long*)it.src, it.n);
      CK(cudaGetLastError());
      ctx->stats.kernel_launches += 1;
    } else {
      std::vector<unsigned long long> tmp(it.n);
      CK(cudaMemcpyAsync(tmp.data(), it.src, it.n * 8, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      unsigned long long* d = (unsigned long long*)it.dst;
      for (size_t i = 0; i < it.n; ++i) d[i] += tmp[i];
    }
  }
  CK(cudaStreamSynchronize(st));
  return KARL_OK;
}

karl_status karl_run(karl_ctx* ctx, const karl_primaries* pr, const karl_run_opts* o,
                     karl_tallies* out) {
  if (!ctx) return KARL_EINVAL;
  ctx->err.clear();
  ctx->drop_retired();
  if (!pr || !out || pr->n < 0) return fail(ctx, KARL_EINVAL, "NULL argument or n < 0");
  karl_status s = check_opts(ctx, o);
  if (s) return s;
  if (o->n_passes != 1 && o->n_passes != 2) return fail(ctx, KARL_EINVAL, "n_passes must be 1 or 2");
  if (!(pr->n_decays > 0)) return fail(ctx, KARL_EINVAL, "n_decays must be > 0");
  if (!out->spectrum || !out->time_fx || !out->cross_pos || !out->cross_neg || !out->recomb ||
      !out->ledger || (ctx->nch > 0 && !out->chan_count))
    return fail(ctx, KARL_EINVAL, "tally buffer is NULL");
  cudaStream_t st = o->stream ? (cudaStream_t)o->stream : ctx->own_stream;
  const double *pz, *pe, *pmu;
  const uint8_t* psp;
  std::memset(ctx->stats.kernel_ms, 0, sizeof ctx->stats.kernel_ms);
  ctx->stats.kernel_launches = 0;
  s = stage_primaries(ctx, pr, st, &pz, &pe, &pmu, &psp);
  if (s) return s;
  bool pp = out->per_primary != nullptr && pr->n > 0;
  s = run_one_pass(ctx, pr, o, 1, pz, pe, pmu, psp, pp, st);
  if (s) return s;
  size_t nt = n_time(ctx);
  CK(ctx->d_time1.ensure(nt));
  CK(cudaMemcpyAsync(ctx->d_time1.p, ctx->d_time.p, nt * 8, cudaMemcpyDeviceToDevice, st));
  if (o->n_passes == 2 && has_recombination(ctx->model)) {
    s = build_fields(ctx, (const unsigned long long*)ctx->d_time1.p, nullptr,
                     (double)pr->n_decays, st);
    if (s) return s;
    s = run_one_pass(ctx, pr, o, 2, pz, pe, pmu, psp, pp, st);
    if (s) return s;
    // the ledger holds pass 2; its all-pass counts take pass 1's as well
    const unsigned long long all[2] = {
        (unsigned long long)(ctx->stats.collisions[0] + ctx->stats.collisions[1]),
        (unsigned long long)(ctx->stats.flights[0] + ctx->stats.flights[1])};
    CK(cudaMemcpyAsync(ctx->d_ledger.p + L_N_COLL_ALL, all, sizeof all, cudaMemcpyHostToDevice,
                       st));
    CK(cudaStreamSynchronize(st));
  }
  // normalisation (Eq. target_field_density, Eq. simulated_time, Sec. 2.3)
  double tsim = (double)pr->n_decays / ctx->activity;
  double vol = ctx->dz * ctx->area;
  CK(ctx->d_density.ensure((size_t)NSP * ctx->nz));
  CK(ctx->d_current.ensure(n_cross(ctx)));
  CK(ctx->d_field.ensure((size_t)NSP * ctx->nz * ctx->ntb));
  k_normalize<<<grid_for(n_cross(ctx), 256), 256, 0, st>>>(
      ctx->d_time.p, (const unsigned long long*)ctx->d_time1.p, ctx->d_recomb.p, ctx->d_cpos.p,
      ctx->d_cneg.p, ctx->d_density.p, ctx->d_current.p, ctx->d_field.p, ctx->nz, ctx->ntb, tsim,
      vol, ctx->area, 0);
  CK(cudaGetLastError());
  ctx->stats.kernel_launches += 1;
  bool dev = out->on_device != 0;
  if ((s = copy_out(ctx, out->spectrum, ctx->d_spec.p, n_spec(ctx) * 8, dev, st)) ||
      (s = copy_out(ctx, out->time_fx, ctx->d_time.p, nt * 8, dev, st)) ||
      (s = copy_out(ctx, out->cross_pos, ctx->d_cpos.p, n_cross(ctx) * 8, dev, st)) ||
      (s = copy_out(ctx, out->cross_neg, ctx->d_cneg.p, n_cross(ctx) * 8, dev, st)) ||
      (s = copy_out(ctx, out->recomb, ctx->d_recomb.p, n_recomb(ctx) * 8, dev, st)) ||
      (s = copy_out(ctx, out->ledger, ctx->d_ledger.p, LEDGER * 8, dev, st)) ||
      (s = copy_out(ctx, out->chan_count, ctx->d_chan.p, (size_t)ctx->nch * 8, dev, st)) ||
      (s = copy_out(ctx, pp ? out->per_primary : nullptr, ctx->d_pp.p, (size_t)pr->n * 8, dev, st)) ||
      (s = copy_out(ctx, out->density, ctx->d_density.p, (size_t)NSP * ctx->nz * 8, dev, st)) ||
      (s = copy_out(ctx, out->current, ctx->d_current.p, n_cross(ctx) * 8, dev, st)) ||
      (s = copy_out(ctx, out->field, ctx->d_field.p, (size_t)NSP * ctx->nz * ctx->ntb * 8, dev, st)))
    return s;
  CK(cudaStreamSynchronize(st));
  return KARL_OK;
}

// Fields of zero for every recombination channel (the first cycle).
karl_status zero_fields(karl_ctx* ctx, cudaStream_t st) {
  size_t nk = (size_t)std::max(ctx->nch, 1);
  CK(ctx->d_frate.ensure(nk * ctx->nz));
  CK(ctx->d_fcol.ensure(nk * (ctx->nz + 1)));
  CK(cudaMemsetAsync(ctx->d_frate.p, 0, nk * ctx->nz * 8, st));
  CK(cudaMemsetAsync(ctx->d_fcol.p, 0, nk * (ctx->nz + 1) * 8, st));
  return KARL_OK;
}

karl_status check_tally_ptrs(karl_ctx* ctx, const karl_tallies* out) {
  if (!out->spectrum || !out->time_fx || !out->cross_pos || !out->cross_neg || !out->recomb ||
      !out->ledger || (ctx->nch > 0 && !out->chan_count))
    return fail(ctx, KARL_EINVAL, "tally buffer is NULL");
  return KARL_OK;
}

karl_status karl_run_cycle(karl_ctx* ctx, const karl_primaries* pr, const karl_run_opts* o,
                           const uint64_t* field_time_in, const uint64_t* field_recomb_in,
                           double field_decays, karl_tallies* out) {
  if (!ctx) return KARL_EINVAL;
  ctx->err.clear();
  ctx->drop_retired();
  if (!pr || !out || pr->n < 0) return fail(ctx, KARL_EINVAL, "NULL argument or n < 0");
  karl_status s = check_opts(ctx, o);
  if (s) return s;
  if (field_time_in && !(field_decays > 0.0) ) return fail(ctx, KARL_EINVAL, "field_decays must be > 0");
  if ((s = check_tally_ptrs(ctx, out))) return s;
  cudaStream_t st = o->stream ? (cudaStream_t)o->stream : ctx->own_stream;
  const double *pz, *pe, *pmu;
  const uint8_t* psp;
  ctx->stats.kernel_launches = 0;
  s = stage_primaries(ctx, pr, st, &pz, &pe, &pmu, &psp);
  if (s) return s;
  if (field_time_in) {
    CK(ctx->d_time1.ensure(n_time(ctx)));
    CK(cudaMemcpyAsync(ctx->d_time1.p, field_time_in, n_time(ctx) * 8, cudaMemcpyHostToDevice, st));
    const unsigned long long* rec = nullptr;
    if (field_recomb_in) {
      CK(ctx->d_recin.ensure(n_recomb(ctx)));
      CK(cudaMemcpyAsync(ctx->d_recin.p, field_recomb_in, n_recomb(ctx) * 8,
                         cudaMemcpyHostToDevice, st));
      rec = ctx->d_recin.p;
    }
    s = build_fields(ctx, (const unsigned long long*)ctx->d_time1.p, rec, field_decays, st);
  } else {
    s = zero_fields(ctx, st);
  }
  if (s) return s;
  bool pp = out->per_primary != nullptr && pr->n > 0;
  s = run_one_pass(ctx, pr, o, 2, pz, pe, pmu, psp, pp, st);
  if (s) return s;
  struct Item { void* dst; const void* src; size_t n; };
  Item items[] = {
      {out->spectrum, ctx->d_spec.p, n_spec(ctx)}, {out->time_fx, ctx->d_time.p, n_time(ctx)},
      {out->cross_pos, ctx->d_cpos.p, n_cross(ctx)}, {out->cross_neg, ctx->d_cneg.p, n_cross(ctx)},
      {out->recomb, ctx->d_recomb.p, n_recomb(ctx)}, {out->ledger, ctx->d_ledger.p, (size_t)LEDGER},
      {out->chan_count, ctx->d_chan.p, (size_t)ctx->nch},
      {pp ? out->per_primary : nullptr, ctx->d_pp.p, (size_t)pr->n}};
  for (const Item& it : items) {
    if (!it.dst || it.n == 0) continue;
    if (out->on_device) {
      k_accumulate<<<grid_for(it.n, 256), 256, 0, st>>>((unsigned long long*)it.dst,
                                                         (const unsigned long long*)it.src, it.n);
      CK(cudaGetLastError());
      ctx->stats.kernel_launches += 1;
    } else {
      std::vector<unsigned long long> tmp(it.n);
      CK(cudaMemcpyAsync(tmp.data(), it.src, it.n * 8, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      unsigned long long* d = (unsigned long long*)it.dst;
      for (size_t i = 0; i < it.n; ++i) d[i] += tmp[i];
    }
  }
  CK(cudaStreamSynchronize(st));
  return KARL_OK;
}

karl_status karl_run_cycles(karl_ctx* ctx, const karl_primaries* pr, const karl_run_opts* o,
                            int32_t n_cycles, karl_tallies* out) {
  if (!ctx) return KARL_EINVAL;
  ctx->err.clear();
  ctx->drop_retired();
  if (!pr || !out || pr->n < 0) return fail(ctx, KARL_EINVAL, "NULL argument or n < 0");
  karl_status s = check_opts(ctx, o);
  if (s) return s;
  if (n_cycles < 1) return fail(ctx, KARL_EINVAL, "n_cycles must be >= 1");
  if (!(pr->n_decays > 0)) return fail(ctx, KARL_EINVAL, "n_decays must be > 0");
  if ((s = check_tally_ptrs(ctx, out))) return s;
  cudaStream_t st = o->stream ? (cudaStream_t)o->stream : ctx->own_stream;
  const double *pz, *pe, *pmu;
  const uint8_t* psp;
  std::memset(ctx->stats.kernel_ms, 0, sizeof ctx->stats.kernel_ms);
  ctx->stats.kernel_launches = 0;
  s = stage_primaries(ctx, pr, st, &pz, &pe, &pmu, &psp);
  if (s) return s;
  const size_t nt = n_time(ctx), nn = (size_t)std::max<int64_t>(pr->n, 1);
  const bool pp = out->per_primary != nullptr && pr->n > 0;
  struct Sum { DevBuf<unsigned long long>* cum; DevBuf<unsigned long long>* one; size_t n; };
  Sum sums[] = {{&ctx->c_spec, &ctx->d_spec, n_spec(ctx)}, {&ctx->c_time, &ctx->d_time, nt},
                {&ctx->c_cpos, &ctx->d_cpos, n_cross(ctx)}, {&ctx->c_cneg, &ctx->d_cneg, n_cross(ctx)},
                {&ctx->c_rec, &ctx->d_recomb, n_recomb(ctx)}, {&ctx->c_led, &ctx->d_ledger, (size_t)LEDGER},
                {&ctx->c_chan, &ctx->d_chan, (size_t)MAXCH}};
  for (Sum& x : sums) {
    CK(x.cum->ensure(x.n));
    CK(cudaMemsetAsync(x.cum->p, 0, x.n * 8, st));
  }
  if (pp) CK(ctx->c_pp.ensure(nn));
  double kms = 0.0;
  int64_t colls = 0, flights = 0, parts = 0;
  const int64_t n = pr->n;
  for (int c = 0; c < n_cycles; ++c) {
    const int64_t lo = n * c / n_cycles, hi = n * (c + 1) / n_cycles;
    if (hi <= lo) continue;
    if (lo == 0) {
      s = zero_fields(ctx, st);
    } else {
      // the fields of every cycle before this one (Sec. 3.6)
      s = build_fields(ctx, ctx->c_time.p, ctx->c_rec.p,
                       (double)pr->n_decays * (double)lo / (double)n, st);
    }
    if (s) return s;
    char name[48];
    snprintf(name, sizeof name, "karl cycle %d", c);
    TraceRange trace(name);
    karl_primaries sl = *pr;
    sl.n = hi - lo;
    sl.pid_offset = pr->pid_offset + lo;
    s = run_one_pass(ctx, &sl, o, 2, pz + lo, pe + lo, pmu + lo, psp + lo, pp, st);
    if (s) return s;
    kms += ctx->stats.kernel_ms[1];
    colls += ctx->stats.collisions[1];
    flights += ctx->stats.flights[1];
    parts += ctx->stats.particles[1];
    for (Sum& x : sums) {
      k_accumulate<<<grid_for(x.n, 256), 256, 0, st>>>(x.cum->p, x.one->p, x.n);
      CK(cudaGetLastError());
      ctx->stats.kernel_launches += 1;
    }
    if (pp) CK(cudaMemcpyAsync(ctx->c_pp.p + lo, ctx->d_pp.p, (size_t)(hi - lo) * 8,
                               cudaMemcpyDeviceToDevice, st));
  }
  ctx->stats.kernel_ms[0] = 0.0;
  ctx->stats.kernel_ms[1] = kms;
  ctx->stats.collisions[0] = 0;
  ctx->stats.collisions[1] = colls;
  ctx->stats.flights[1] = flights;
  ctx->stats.particles[1] = parts;
  // normalisation over the whole run (Eq. target_field_density, Sec. 2.3)
  const double tsim = (double)pr->n_decays / ctx->activity;
  const double vol = ctx->dz * ctx->area;
  CK(ctx->d_density.ensure((size_t)NSP * ctx->nz));
  CK(ctx->d_current.ensure(n_cross(ctx)));
  CK(ctx->d_field.ensure((size_t)NSP * ctx->nz * ctx->ntb));
  k_normalize<<<grid_for(n_cross(ctx), 256), 256, 0, st>>>(
      ctx->c_time.p, ctx->c_time.p, ctx->c_rec.p, ctx->c_cpos.p, ctx->c_cneg.p, ctx->d_density.p,
      ctx->d_current.p, ctx->d_field.p, ctx->nz, ctx->ntb, tsim, vol, ctx->area, 1);
  CK(cudaGetLastError());
  ctx->stats.kernel_launches += 1;
  const bool dev = out->on_device != 0;
  if ((s = copy_out(ctx, out->spectrum, ctx->c_spec.p, n_spec(ctx) * 8, dev, st)) ||
      (s = copy_out(ctx, out->time_fx, ctx->c_time.p, nt * 8, dev, st)) ||
      (s = copy_out(ctx, out->cross_pos, ctx->c_cpos.p, n_cross(ctx) * 8, dev, st)) ||
      (s = copy_out(ctx, out->cross_neg, ctx->c_cneg.p, n_cross(ctx) * 8, dev, st)) ||
      (s = copy_out(ctx, out->recomb, ctx->c_rec.p, n_recomb(ctx) * 8, dev, st)) ||
      (s = copy_out(ctx, out->ledger, ctx->c_led.p, LEDGER * 8, dev, st)) ||
      (s = copy_out(ctx, out->chan_count, ctx->c_chan.p, (size_t)ctx->nch * 8, dev, st)) ||
      (s = copy_out(ctx, pp ? out->per_primary : nullptr, ctx->c_pp.p, (size_t)n * 8, dev, st)) ||
      (s = copy_out(ctx, out->density, ctx->d_density.p, (size_t)NSP * ctx->nz * 8, dev, st)) ||
      (s = copy_out(ctx, out->current, ctx->d_current.p, n_cross(ctx) * 8, dev, st)) ||
      (s = copy_out(ctx, out->field, ctx->d_field.p, (size_t)NSP * ctx->nz * ctx->ntb * 8, dev, st)))
    return s;
  CK(cudaStreamSynchronize(st));
  return KARL_OK;
}

void karl_destroy(karl_ctx* ctx) {
  if (!ctx) return;
  if (ctx->own_stream) cudaStreamSynchronize(ctx->own_stream);
  int prev = -1;
  if (cudaGetDevice(&prev) == cudaSuccess && prev != ctx->device) cudaSetDevice(ctx->device);
  ctx->each_buf([](auto& b) { b.release(); });
  ctx->d_ctl = nullptr;
  ctx->d_cancel = nullptr;
  if (ctx->cancel_stream) cudaStreamDestroy(ctx->cancel_stream);
  if (ctx->ev0) cudaEventDestroy(ctx->ev0);
  if (ctx->ev1) cudaEventDestroy(ctx->ev1);
  if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
  if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
  delete ctx;
}

}  // extern "C"

// ===========================================================================
// One pass with no allocation: all scratch in one static device array.
//
// For callers that must not allocate device memory while they run (a caching
// allocator or a fixed memory budget that reserves the GPU up front, or a
// request path that keeps allocation out).  The transport kernel is the same
// as karl_run_pass's; only where its scratch lives differs.  The array is
// carried by the library image: the CUDA runtime maps it when the module is
// loaded on a device, before any call, and this code only looks up its
// address.

// KARL_STATIC_SCRATCH_BYTES of scratch per device, 256-byte aligned so every
// region carved from it keeps the alignment of its element type.
static __device__ __align__(256) unsigned char karl_static_scratch[KARL_STATIC_SCRATCH_BYTES];

namespace {

constexpr int SCRATCH_MAX_DEVICES = 64;
constexpr unsigned long long SCRATCH_RING_MIN = 1ULL << 16;   // particles
constexpr unsigned long long SCRATCH_RING_MAX = 1ULL << 19;   // 32 MiB of 64-byte cells

std::mutex g_scratch_mu;
unsigned char* g_scratch_addr[SCRATCH_MAX_DEVICES];           // zero-initialised
bool g_scratch_ready[SCRATCH_MAX_DEVICES];

// Device address of the static scratch on ctx->device, looked up the first
// time with that device current.  Later calls reuse it.
karl_status static_scratch(karl_ctx* ctx, unsigned char** out) {
  if (ctx->device < 0 || ctx->device >= SCRATCH_MAX_DEVICES)
    return fail(ctx, KARL_EINVAL, "device %d beyond the static scratch table", ctx->device);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ready[ctx->device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, karl_static_scratch);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGetSymbolAddress(karl_static_scratch)");
    if (!p) return fail(ctx, KARL_ECUDA, "static scratch has no device address");
    g_scratch_addr[ctx->device] = (unsigned char*)p;
    g_scratch_ready[ctx->device] = true;
  }
  *out = g_scratch_addr[ctx->device];
  return KARL_OK;
}

// Bump allocator over the static array (256-byte regions, no device call).
struct Carve {
  unsigned char* base;
  size_t used = 0;
  template <class T>
  T* take(size_t count) {
    T* p = (T*)(base + used);
    used += (count * sizeof(T) + 255) & ~(size_t)255;
    return p;
  }
};

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// A pointer the kernels may dereference on ctx->device: device memory (or
// managed memory) of that device.  cudaPointerGetAttributes allocates
// nothing; a host array passed here would otherwise be read by a kernel.
karl_status check_device_ptr(karl_ctx* ctx, const void* p, const char* what) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();                           // clear the sticky-free error state
    return fail(ctx, KARL_EINVAL, "%s: not a CUDA device pointer", what);
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
    return fail(ctx, KARL_EINVAL, "%s: host memory; karl_run_pass_static reads device memory only",
                what);
  if (a.type == cudaMemoryTypeDevice && a.device != ctx->device)
    return fail(ctx, KARL_EINVAL, "%s: memory of device %d, the context is on device %d", what,
                a.device, ctx->device);
  return KARL_OK;
}

// z eq mu node tal pid seq (8 bytes each), ev sj (4 bytes each) per ring cell
size_t ring_bytes(unsigned long long cap) {
  return 7 * round256((size_t)cap * 8) + 2 * round256((size_t)cap * 4);
}

}  // namespace

extern "C" karl_status karl_run_pass_static(karl_ctx* ctx, const karl_primaries* pr,
                                            const karl_run_opts* o, int32_t pass,
                                            const uint64_t* field_time_in, karl_tallies* out) {
  if (!ctx) return KARL_EINVAL;
  ctx->err.clear();
  if (!pr || !out || pr->n < 0) return fail(ctx, KARL_EINVAL, "NULL argument or n < 0");
  karl_status s = check_opts(ctx, o);
  if (s) return s;
  if (pass != 1 && pass != 2) return fail(ctx, KARL_EINVAL, "pass must be 1 or 2");
  if (pass == 2 && !field_time_in) return fail(ctx, KARL_EINVAL, "pass 2 needs field_time_in");
  if (pass == 2 && !(pr->n_decays > 0)) return fail(ctx, KARL_EINVAL, "n_decays must be > 0");
  if (!pr->on_device || !out->on_device)
    return fail(ctx, KARL_EINVAL, "karl_run_pass_static takes device primaries and tallies only");
  if (pr->n > 0 && (!pr->z_m || !pr->e_ev || !pr->mu || !pr->species))
    return fail(ctx, KARL_EINVAL, "primaries: NULL array");
  if (!out->spectrum || !out->time_fx || !out->cross_pos || !out->cross_neg || !out->recomb ||
      !out->ledger || (ctx->nch > 0 && !out->chan_count))
    return fail(ctx, KARL_EINVAL, "tally buffer is NULL");
  // every array the kernels touch must be memory of this context's device
  {
    const struct { const void* p; const char* what; bool need; } ptrs[] = {
        {pr->z_m, "primaries z_m", pr->n > 0}, {pr->e_ev, "primaries e_ev", pr->n > 0},
        {pr->mu, "primaries mu", pr->n > 0}, {pr->species, "primaries species", pr->n > 0},
        {out->spectrum, "tallies spectrum", true}, {out->time_fx, "tallies time_fx", true},
        {out->cross_pos, "tallies cross_pos", true}, {out->cross_neg, "tallies cross_neg", true},
        {out->recomb, "tallies recomb", true}, {out->ledger, "tallies ledger", true},
        {out->chan_count, "tallies chan_count", ctx->nch > 0},
        {out->per_primary, "tallies per_primary", out->per_primary != nullptr && pr->n > 0},
        {field_time_in, "field_time_in", pass == 2}};
    for (const auto& q : ptrs)
      if (q.need && (s = check_device_ptr(ctx, q.p, q.what)) != KARL_OK) return s;
  }

  // the scratch plan, checked before any device call
  const size_t nt = n_time(ctx), nx = n_cross_rg(ctx);
  const size_t nk = (size_t)std::max(ctx->nch, 1);
  size_t fixed = round256(sizeof(Control)) + round256(sizeof(int)) + 2 * round256(nt * 8) +
                 2 * round256(nx * 8);
  if (pass == 2) fixed += round256(nk * ctx->nz * 8) + round256(nk * (ctx->nz + 1) * 8);
  const size_t total = KARL_STATIC_SCRATCH_BYTES;
  if (fixed + ring_bytes(SCRATCH_RING_MIN) > total)
    return fail(ctx, KARL_ECAPACITY,
                "problem needs %zu bytes of scratch (tallies %zu + particle ring %zu); the "
                "static scratch holds %zu",
                fixed + ring_bytes(SCRATCH_RING_MIN), fixed, ring_bytes(SCRATCH_RING_MIN), total);
  unsigned long long cap = SCRATCH_RING_MIN;
  while (cap < SCRATCH_RING_MAX && fixed + ring_bytes(cap * 2) <= total) cap *= 2;

  int prev_dev = -1;
  if (cudaGetDevice(&prev_dev) != cudaSuccess) return fail(ctx, KARL_ECUDA, "cudaGetDevice failed");
  if (prev_dev != ctx->device) CK(cudaSetDevice(ctx->device));
  struct Restore {
    int d, want;
    ~Restore() { if (d >= 0 && d != want) cudaSetDevice(d); }
  } restore{prev_dev, ctx->device};

  unsigned char* base = nullptr;
  s = static_scratch(ctx, &base);
  if (s) return s;
  Carve cv{base};
  Control* ctl = cv.take<Control>(1);
  int* bad = cv.take<int>(1);
  unsigned long long* tpt = cv.take<unsigned long long>(nt);
  unsigned long long* trg = cv.take<unsigned long long>(nt);
  unsigned long long* xpos = cv.take<unsigned long long>(nx);
  unsigned long long* xneg = cv.take<unsigned long long>(nx);
  double* frate = pass == 2 ? cv.take<double>(nk * ctx->nz) : nullptr;
  double* fcol = pass == 2 ? cv.take<double>(nk * (ctx->nz + 1)) : nullptr;
  Ring R;
  R.z = cv.take<double>(cap); R.eq = cv.take<long long>(cap); R.mu = cv.take<double>(cap);
  R.node = cv.take<unsigned long long>(cap); R.tal = cv.take<double>(cap);
  R.pid = cv.take<unsigned long long>(cap); R.seq = cv.take<unsigned long long>(cap);
  R.ev = cv.take<unsigned>(cap); R.sj = cv.take<unsigned>(cap);
  R.cap = cap; R.mask = cap - 1;
  if (cv.used > total) return fail(ctx, KARL_ECAPACITY, "static scratch plan overran");

  cudaStream_t st = o->stream ? (cudaStream_t)o->stream : ctx->own_stream;
  ctx->stats.kernel_launches = 0;
  const size_t n = (size_t)pr->n;

  // what must start at zero: the control block, the primary check counter,
  // the difference arrays, and every caller tally the kernel adds into
  CK(cudaMemsetAsync(ctl, 0, sizeof(Control), st));
  CK(cudaMemsetAsync(bad, 0, sizeof(int), st));
  CK(cudaMemsetAsync(tpt, 0, nt * 8, st));
  CK(cudaMemsetAsync(trg, 0, nt * 8, st));
  CK(cudaMemsetAsync(xpos, 0, nx * 8, st));
  CK(cudaMemsetAsync(xneg, 0, nx * 8, st));
  CK(cudaMemsetAsync(out->spectrum, 0, n_spec(ctx) * 8, st));
  CK(cudaMemsetAsync(out->recomb, 0, n_recomb(ctx) * 8, st));
  CK(cudaMemsetAsync(out->ledger, 0, LEDGER * 8, st));
  if (ctx->nch > 0) CK(cudaMemsetAsync(out->chan_count, 0, (size_t)ctx->nch * 8, st));
  const bool pp = out->per_primary != nullptr && n > 0;
  if (pp) CK(cudaMemsetAsync(out->per_primary, 0, n * 8, st));
  k_ring_init<<<grid_for((size_t)cap, 256), 256, 0, st>>>(R.seq, cap);
  CK(cudaGetLastError());
  ctx->stats.kernel_launches += 1;

  if (n > 0) {
    k_check_primaries<<<grid_for(n, 256), 256, 0, st>>>(pr->z_m, pr->e_ev, pr->mu, pr->species,
                                                        (long long)n, ctx->L, bad);
    CK(cudaGetLastError());
    ctx->stats.kernel_launches += 1;
    int hbad = 0;
    CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (hbad) return fail(ctx, KARL_EINVAL, "%d primaries out of range", hbad);
  }

  Params P;
  base_params(ctx, P, o, pass);
  if (pass == 2) {
    FieldArgs A;
    std::memset(&A, 0, sizeof A);
    A.nz = ctx->nz; A.ntb = ctx->ntb; A.n_energy = ctx->n_energy; A.nch = ctx->nch;
    A.tsim = (double)pr->n_decays / ctx->activity;
    A.vol = ctx->dz * ctx->area;
    A.dz = ctx->dz; A.e_min = ctx->e_min; A.e_max = ctx->e_max; A.me = ctx->mass[SP_E];
    for (int k = 0; k < ctx->nch; ++k) {
      A.kind[k] = ctx->kind[k]; A.sin[k] = ctx->sin[k];
      A.sout[k] = ctx->sout[k]; A.loss[k] = ctx->loss[k];
    }
    CK(cudaMemsetAsync(frate, 0, nk * ctx->nz * 8, st));
    k_build_fields<<<grid_for((size_t)ctx->nch * ctx->nz, 256), 256, 0, st>>>(
        A, (const unsigned long long*)field_time_in, nullptr, ctx->d_sig.p, frate, fcol);
    k_field_columns<<<1, 32, 0, st>>>(frate, fcol, ctx->nch, ctx->nz, ctx->dz);
    CK(cudaGetLastError());
    ctx->stats.kernel_launches += 2;
    for (int k = 0; k < ctx->nch; ++k) {
      if (ctx->kind[k] != RECOMBINATION) continue;
      P.frate[k] = frate + (size_t)k * ctx->nz;
      P.fcol[k] = fcol + (size_t)k * (ctx->nz + 1);
    }
  }
  P.pid_offset = pr->pid_offset;
  P.n_prim = pr->n;
  P.pz = pr->z_m; P.pe = pr->e_ev; P.pmu = pr->mu; P.psp = pr->species;
  P.spectrum = (unsigned long long*)out->spectrum;
  P.time_pt = tpt;
  P.time_rg = trg;
  P.xpos_rg = xpos;
  P.xneg_rg = xneg;
  P.recomb = (unsigned long long*)out->recomb;
  P.ledger = (unsigned long long*)out->ledger;
  P.chan_count = (unsigned long long*)out->chan_count;
  P.per_primary = pp ? (unsigned long long*)out->per_primary : nullptr;

  const bool f32 = o->precision == KARL_FP32;
  const int block = o->block_size > 0 ? o->block_size : default_block(f32);
  int bps = 0;
  CK(transport_occupancy(f32, P, block, &bps));
  if (o->blocks_per_sm > 0) bps = std::min(bps, (int)o->blocks_per_sm);
  if (bps < 1) bps = 1;
  const int grid = ctx->num_sms * bps;
  const double timeout = o->timeout_s > 0 ? o->timeout_s : 600.0;

  CK(cudaMemsetAsync(ctx->d_cancel, 0, sizeof(int), st));
  CK(cudaEventRecord(ctx->ev0, st));
  CK(launch_transport(f32, P, R, ctl, ctx->d_cancel, (unsigned long long)(timeout * 1e9), grid,
                      block, st));
  CK(cudaEventRecord(ctx->ev1, st));
  ctx->stats.kernel_launches += 1;
  k_finalize_time<<<grid_for((size_t)NSP * ctx->ntb, 64), 64, 0, st>>>(
      tpt, trg, (unsigned long long*)out->time_fx, ctx->nz, ctx->ntb);
  k_finalize_cross<<<1, 32, 0, st>>>(xpos, (unsigned long long*)out->cross_pos, ctx->nz);
  k_finalize_cross<<<1, 32, 0, st>>>(xneg, (unsigned long long*)out->cross_neg, ctx->nz);
  CK(cudaGetLastError());
  ctx->stats.kernel_launches += 3;
  Control hc;
  CK(cudaMemcpyAsync(&hc, ctl, sizeof hc, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));

  float ms = 0;
  cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
  const int pi = pass - 1;
  ctx->stats.kernel_ms[pi] = ms;
  ctx->stats.particles[pi] = (int64_t)hc.particles;
  ctx->stats.spilled[pi] = (int64_t)hc.spilled;
  ctx->stats.idle_warp_frac[pi] =
      hc.busy_iters + hc.idle_iters
          ? (double)hc.idle_iters / (double)(hc.busy_iters + hc.idle_iters)
          : 0.0;
  ctx->stats.tail_ms[pi] =
      hc.t_end > hc.t_claimed && hc.t_claimed ? (double)(hc.t_end - hc.t_claimed) * 1e-6 : 0.0;
  ctx->stats.lane_occupancy[pi] =
      hc.busy_iters + hc.idle_iters
          ? (double)hc.busy_lane_iters / (32.0 * (double)(hc.busy_iters + hc.idle_iters))
          : 0.0;
  ctx->stats.grid_blocks = grid;
  ctx->stats.block_size = block;
  ctx->stats.queue_capacity = (int32_t)cap;
  if (hc.error == ERR_CAPACITY)
    return fail(ctx, KARL_ECAPACITY,
                "particle ring overflow at its static capacity %llu (the ring cannot grow; use "
                "karl_run_pass, or fewer primaries per call)",
                (unsigned long long)cap);
  if (hc.error == ERR_TIMEOUT) return fail(ctx, KARL_ETIMEOUT, "transport kernel timed out");
  if (hc.error == ERR_CANCELLED) return fail(ctx, KARL_ECANCELLED, "run cancelled");
  if (hc.error != 0) return fail(ctx, KARL_ECUDA, "transport kernel error %d", hc.error);
  long long led[LEDGER];
  CK(cudaMemcpyAsync(led, out->ledger, sizeof led, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  ctx->stats.collisions[pi] = led[L_N_COLL];
  ctx->stats.flights[pi] = led[L_N_FLIGHT];
  return KARL_OK;
}

// ===========================================================================
// Full-orbit transport (Sec. 3.1 Boris mover): one launch per generation of
// particles, the products of one generation being the next one's list.

namespace {

constexpr double ORBIT_CHARGE[NSP] = {-1.0, 1.0, 1.0, 1.0};   // units of e
constexpr int ORBIT_MAX_GENERATIONS = 4096;

karl_status check_orbit(karl_ctx* ctx, const karl_orbit* ob, const karl_orbit_primaries* pr,
                        const karl_run_opts* o, const karl_orbit_tallies* out) {
  if (!ob || !pr || !o || !out) return fail(ctx, KARL_EINVAL, "NULL argument");
  if (o->precision != KARL_FP64) return fail(ctx, KARL_EINVAL, "orbit runs are FP64 only");
  if (o->block_size != 0 && (o->block_size < 32 || o->block_size > 256 || o->block_size % 32))
    return fail(ctx, KARL_EINVAL, "block_size must be a multiple of 32 in [32, 256]");
  if (!std::isfinite(ob->b_t) || !(ob->tube_radius_m > 0.0) || !std::isfinite(ob->tube_radius_m) ||
      ob->n_rbins < 1 || ob->n_rbins > (1 << 20) || !std::isfinite(ob->e_r_vm2))
    return fail(ctx, KARL_EINVAL, "invalid orbit field, radius or radial bins");
  for (int s = 0; s < NSP; ++s)
    if (!(ob->dt_s[s] > 0.0) || !std::isfinite(ob->dt_s[s]))
      return fail(ctx, KARL_EINVAL, "time step of species %d must be positive", s);
  if (ob->e_z_vm)
    for (int j = 0; j < ctx->nz; ++j)
      if (!std::isfinite(ob->e_z_vm[j])) return fail(ctx, KARL_EINVAL, "e_z_vm[%d] not finite", j);
  for (int k = 0; k < ctx->nch; ++k) {
    const int kd = ctx->kind[k];
    if (kd == RECOMBINATION || kd == CHARGE_EXCHANGE)
      return fail(ctx, KARL_EINVAL, "channel %d: kind %d is not available in orbit runs", k, kd);
    if ((kd == ELASTIC || kd == IONIZATION) && ctx->model.target[k] != 0)
      return fail(ctx, KARL_EINVAL, "channel %d: moving targets are not available in orbit runs", k);
  }
  if (pr->n < 0) return fail(ctx, KARL_EINVAL, "n < 0");
  if (pr->n > 0 && (!pr->x_m || !pr->y_m || !pr->z_m || !pr->e_ev || !pr->mu || !pr->phi ||
                    !pr->species))
    return fail(ctx, KARL_EINVAL, "primary array is NULL");
  const double R2 = ob->tube_radius_m * ob->tube_radius_m;
  for (int64_t i = 0; i < pr->n; ++i) {
    const double x = pr->x_m[i], y = pr->y_m[i], z = pr->z_m[i];
    if (!(x * x + y * y < R2) || !(z >= 0.0 && z <= ctx->L) || pr->species[i] >= NSP ||
        !(pr->e_ev[i] >= 0.0) || !std::isfinite(pr->e_ev[i]) || !(std::fabs(pr->mu[i]) <= 1.0) ||
        !std::isfinite(pr->phi[i]))
      return fail(ctx, KARL_EINVAL, "primary %lld outside the tube or invalid", (long long)i);
  }
  if (!out->spectrum || !out->time_z || !out->time_r || !out->cross_pos || !out->cross_neg ||
      !out->rcross_out || !out->rcross_in || !out->wall || !out->ledger || !out->energy ||
      (ctx->nch > 0 && !out->chan_count))
    return fail(ctx, KARL_EINVAL, "tally buffer is NULL");
  return KARL_OK;
}

// Host buffer `src` of n elements into device buffer b (n may be 0).
template <class T>
karl_status upload(karl_ctx* ctx, DevBuf<T>& b, const T* src, size_t n, cudaStream_t st) {
  CK(b.ensure(n));
  if (n) CK(cudaMemcpyAsync(b.p, src, n * sizeof(T), cudaMemcpyHostToDevice, st));
  return KARL_OK;
}

template <class T>
karl_status zeroed(karl_ctx* ctx, DevBuf<T>& b, size_t n, cudaStream_t st) {
  CK(b.ensure(n));
  CK(cudaMemsetAsync(b.p, 0, std::max<size_t>(n, 1) * sizeof(T), st));
  return KARL_OK;
}

// Add device buffer b (n u64) into the host buffer dst.
karl_status add_out(karl_ctx* ctx, const DevBuf<unsigned long long>& b, uint64_t* dst, size_t n,
                    cudaStream_t st) {
  if (!dst || !n) return KARL_OK;
  std::vector<unsigned long long> h(n);
  CK(cudaMemcpyAsync(h.data(), b.p, n * 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (size_t i = 0; i < n; ++i) dst[i] += h[i];
  return KARL_OK;
}

karl_status ensure_list(karl_ctx* ctx, int g, size_t n) {
  CK(ctx->o_lx[g].ensure(n)); CK(ctx->o_ly[g].ensure(n)); CK(ctx->o_lz[g].ensure(n));
  CK(ctx->o_lux[g].ensure(n)); CK(ctx->o_luy[g].ensure(n)); CK(ctx->o_luz[g].ensure(n));
  CK(ctx->o_lnode[g].ensure(n)); CK(ctx->o_lpid[g].ensure(n)); CK(ctx->o_lsp[g].ensure(n));
  return KARL_OK;
}

OrbitList list_of(karl_ctx* ctx, int g) {
  OrbitList L;
  L.x = ctx->o_lx[g].p; L.y = ctx->o_ly[g].p; L.z = ctx->o_lz[g].p;
  L.ux = ctx->o_lux[g].p; L.uy = ctx->o_luy[g].p; L.uz = ctx->o_luz[g].p;
  L.node = ctx->o_lnode[g].p; L.pid = ctx->o_lpid[g].p; L.sp = ctx->o_lsp[g].p;
  return L;
}

}  // namespace

extern "C" karl_status karl_run_orbit(karl_ctx* ctx, const karl_orbit* ob,
                                      const karl_orbit_primaries* pr, const karl_run_opts* o,
                                      karl_orbit_tallies* out) {
  if (!ctx) return KARL_EINVAL;
  ctx->err.clear();
  ctx->drop_retired();
  karl_status s = check_orbit(ctx, ob, pr, o, out);
  if (s) return s;
  TraceRange trace("karl orbit run");
  cudaStream_t st = o->stream ? (cudaStream_t)o->stream : ctx->own_stream;
  const size_t n = (size_t)pr->n, nz = (size_t)ctx->nz, nr = (size_t)ob->n_rbins;
  std::memset(ctx->stats.kernel_ms, 0, sizeof ctx->stats.kernel_ms);
  ctx->stats.kernel_launches = 0;
  if ((s = upload(ctx, ctx->o_px, pr->x_m, n, st)) || (s = upload(ctx, ctx->o_py, pr->y_m, n, st)) ||
      (s = upload(ctx, ctx->o_pz, pr->z_m, n, st)) || (s = upload(ctx, ctx->o_pe, pr->e_ev, n, st)) ||
      (s = upload(ctx, ctx->o_pmu, pr->mu, n, st)) ||
      (s = upload(ctx, ctx->o_pphi, pr->phi, n, st)) ||
      (s = upload(ctx, ctx->o_psp, pr->species, n, st)) ||
      (s = upload(ctx, ctx->o_ez, ob->e_z_vm, ob->e_z_vm ? nz : 0, st)))
    return s;
  const size_t nspec = n_spec(ctx), ncross = nz + 1;
  if ((s = zeroed(ctx, ctx->o_tz, NSP * nz, st)) || (s = zeroed(ctx, ctx->o_tr, NSP * nr, st)) ||
      (s = zeroed(ctx, ctx->o_xp, NSP * ncross, st)) ||
      (s = zeroed(ctx, ctx->o_xn, NSP * ncross, st)) ||
      (s = zeroed(ctx, ctx->o_ro, NSP * (nr + 1), st)) ||
      (s = zeroed(ctx, ctx->o_ri, NSP * (nr + 1), st)) ||
      (s = zeroed(ctx, ctx->o_wall, NSP * nz, st)) || (s = zeroed(ctx, ctx->o_spec, nspec, st)) ||
      (s = zeroed(ctx, ctx->o_led, (size_t)KARL_ORBIT_LEDGER, st)) ||
      (s = zeroed(ctx, ctx->o_chan, (size_t)std::max(ctx->nch, 1), st)) ||
      (s = zeroed(ctx, ctx->o_energy, (size_t)KARL_ORBIT_ENERGY, st)) ||
      (s = zeroed(ctx, ctx->o_pp, out->per_primary ? n : 0, st)) ||
      (s = zeroed(ctx, ctx->o_end, out->end_state ? 8 * n : 0, st)) ||
      (s = zeroed(ctx, ctx->o_cnt, 2, st)) || (s = zeroed(ctx, ctx->o_err, 1, st)))
    return s;

  Params P;
  karl_run_opts o1 = *o;
  o1.n_passes = 1;
  base_params(ctx, P, &o1, 1);
  P.pid_offset = pr->pid_offset;
  OrbitDev O;
  std::memset(&O, 0, sizeof O);
  O.bz = ob->b_t;
  O.R2 = ob->tube_radius_m * ob->tube_radius_m;
  O.r_scale = (double)ob->n_rbins / ob->tube_radius_m;
  O.er = ob->e_r_vm2;
  for (int sp = 0; sp < NSP; ++sp) {
    O.dt[sp] = ob->dt_s[sp];
    O.h[sp] = 0.5 * (ORBIT_CHARGE[sp] * C_LIGHT * C_LIGHT / ctx->mass[sp]) * ob->dt_s[sp];
  }
  O.e_cut = ctx->e_cut;
  O.spec_bin = ctx->spec_bin;
  O.inv_dz = (double)ctx->nz / ctx->L;
  O.e_max = ctx->e_max;
  // u^2 = (gamma v)^2 at the edges of the energy grid's bins, per species
  {
    const int ntb = ctx->ntb;
    std::vector<double> edge((size_t)NSP * (ntb + 1));
    const double ratio = ctx->e_max / ctx->e_min;
    for (int sp = 0; sp < NSP; ++sp)
      for (int k = 0; k <= ntb; ++k) {
        const double y = ctx->e_min * std::pow(ratio, (double)k / ntb) / ctx->mass[sp];
        const double ps = C_LIGHT * std::sqrt(y * (2.0 + y));
        edge[(size_t)sp * (ntb + 1) + k] = ps * ps;
      }
    if ((s = upload(ctx, ctx->o_u2edge, edge.data(), edge.size(), st))) return s;
    O.u2edge = ctx->o_u2edge.p;
    // squared radii of the radial bin edges
    std::vector<double> e2((size_t)ob->n_rbins + 1);
    for (int k = 0; k <= ob->n_rbins; ++k) {
      const double rk = ob->tube_radius_m * (double)k / (double)ob->n_rbins;
      e2[k] = rk * rk;
    }
    if ((s = upload(ctx, ctx->o_edge2, e2.data(), e2.size(), st))) return s;
    O.edge2 = ctx->o_edge2.p;
    CK(cudaStreamSynchronize(st));        // the host tables above go out of scope
  }
  O.ez = ob->e_z_vm ? ctx->o_ez.p : nullptr;
  O.nr = ob->n_rbins;
  O.fields = ob->e_r_vm2 != 0.0;
  if (ob->e_z_vm)
    for (size_t j = 0; j < nz; ++j) O.fields = O.fields || ob->e_z_vm[j] != 0.0;
  O.max_steps = ob->max_steps ? ob->max_steps : (1ULL << 40);
  O.px = ctx->o_px.p; O.py = ctx->o_py.p; O.pz = ctx->o_pz.p; O.pe = ctx->o_pe.p;
  O.pmu = ctx->o_pmu.p; O.pphi = ctx->o_pphi.p; O.psp = ctx->o_psp.p;
  O.counters = ctx->o_cnt.p;
  O.time_z = ctx->o_tz.p; O.time_r = ctx->o_tr.p; O.xpos = ctx->o_xp.p; O.xneg = ctx->o_xn.p;
  O.rout = ctx->o_ro.p; O.rin = ctx->o_ri.p; O.wall = ctx->o_wall.p; O.spectrum = ctx->o_spec.p;
  O.ledger = ctx->o_led.p; O.chan = ctx->o_chan.p;
  O.per_primary = out->per_primary ? ctx->o_pp.p : nullptr;
  O.energy = ctx->o_energy.p;
  O.end_state = out->end_state ? ctx->o_end.p : nullptr;
  O.error = ctx->o_err.p;
  O.cancel = ctx->d_cancel;
  const double timeout = o->timeout_s > 0 ? o->timeout_s : 600.0;
  O.timeout_ns = (unsigned long long)(timeout * 1e9);

  const int block = o->block_size > 0 ? o->block_size : 256;
  int bps = 0;
  CK(orbit_occupancy(block, &bps));
  if (o->blocks_per_sm > 0) bps = std::min(bps, (int)o->blocks_per_sm);
  if (bps < 1) bps = 1;
  const int grid = ctx->num_sms * bps;
  CK(cudaMemsetAsync(ctx->d_cancel, 0, sizeof(int), st));

  long long n_in = (long long)n;
  int cur = 0;                                        // list holding the current generation
  float total_ms = 0.0f;
  for (int gen = 0; n_in > 0; ++gen) {
    if (gen >= ORBIT_MAX_GENERATIONS)
      return fail(ctx, KARL_ECAPACITY, "more than %d product generations", ORBIT_MAX_GENERATIONS);
    const unsigned long long cap =
        std::max<unsigned long long>(1ULL << 20, 8ULL * (unsigned long long)n_in);
    if ((s = ensure_list(ctx, 1 - cur, (size_t)cap))) return s;
    if (gen > 0 && (s = ensure_list(ctx, cur, (size_t)n_in))) return s;
    O.from_primaries = gen == 0;
    O.n_in = n_in;
    O.in = list_of(ctx, cur);
    O.out = list_of(ctx, 1 - cur);
    O.out_cap = cap;
    CK(cudaMemsetAsync(ctx->o_cnt.p, 0, 2 * sizeof(unsigned long long), st));
    CK(cudaEventRecord(ctx->ev0, st));
    CK(launch_orbit(P, O, grid, block, st));
    CK(cudaEventRecord(ctx->ev1, st));
    unsigned long long cnt[2] = {0, 0};
    int err = 0;
    CK(cudaMemcpyAsync(cnt, ctx->o_cnt.p, sizeof cnt, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&err, ctx->o_err.p, sizeof err, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    total_ms += ms;
    ctx->stats.kernel_launches += 1;
    if (err == ERR_CAPACITY)
      return fail(ctx, KARL_ECAPACITY, "generation %d: more than %llu products", gen, cap);
    if (err == ERR_TIMEOUT) return fail(ctx, KARL_ETIMEOUT, "orbit kernel timed out");
    if (err == ERR_CANCELLED) return fail(ctx, KARL_ECANCELLED, "run cancelled");
    if (err != 0) return fail(ctx, KARL_ECUDA, "orbit kernel error %d", err);
    n_in = (long long)cnt[1];
    cur = 1 - cur;
  }
  ctx->stats.kernel_ms[0] = total_ms;
  ctx->stats.grid_blocks = grid;
  ctx->stats.block_size = block;
  if ((s = add_out(ctx, ctx->o_spec, out->spectrum, nspec, st)) ||
      (s = add_out(ctx, ctx->o_tz, out->time_z, NSP * nz, st)) ||
      (s = add_out(ctx, ctx->o_tr, out->time_r, NSP * nr, st)) ||
      (s = add_out(ctx, ctx->o_xp, out->cross_pos, NSP * ncross, st)) ||
      (s = add_out(ctx, ctx->o_xn, out->cross_neg, NSP * ncross, st)) ||
      (s = add_out(ctx, ctx->o_ro, out->rcross_out, NSP * (nr + 1), st)) ||
      (s = add_out(ctx, ctx->o_ri, out->rcross_in, NSP * (nr + 1), st)) ||
      (s = add_out(ctx, ctx->o_wall, out->wall, NSP * nz, st)) ||
      (s = add_out(ctx, ctx->o_led, (uint64_t*)out->ledger, (size_t)KARL_ORBIT_LEDGER, st)) ||
      (s = add_out(ctx, ctx->o_chan, out->chan_count, (size_t)ctx->nch, st)) ||
      (s = add_out(ctx, ctx->o_pp, out->per_primary, out->per_primary ? n : 0, st)))
    return s;
  std::vector<double> e(KARL_ORBIT_ENERGY);
  CK(cudaMemcpyAsync(e.data(), ctx->o_energy.p, e.size() * 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int i = 0; i < KARL_ORBIT_ENERGY; ++i) out->energy[i] += e[i];
  if (out->end_state && n) {
    CK(cudaMemcpyAsync(out->end_state, ctx->o_end.p, 8 * n * sizeof(double),
                       cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  long long led[KARL_ORBIT_LEDGER];
  CK(cudaMemcpy(led, ctx->o_led.p, sizeof led, cudaMemcpyDeviceToHost));
  ctx->stats.collisions[0] = led[OB_N_COLL];
  ctx->stats.flights[0] = led[OB_N_FLIGHT];
  ctx->stats.particles[0] = led[OB_BIRTHS] + led[OB_BIRTHS + 1] + led[OB_BIRTHS + 2] +
                            led[OB_BIRTHS + 3];
  return KARL_OK;
}
