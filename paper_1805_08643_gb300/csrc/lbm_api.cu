// C ABI of the library (declared in include/lbm.h): context lifetime, device
// buffers, initial states, the time-step loop, observables and reductions.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

using lbm::KParams;

namespace lbm {
bool fill_params(const int grid[3], const lbm_eos *eos, double G, const lbm_rates *rates, int op, int precision,
                 double sigma, KParams *out);
}

struct lbm_ctx {
  KParams P{};
  int precision = 0, op = 1;
  bool sigma_on = false;
  lbm::Launch L{};
  void *g[2] = {nullptr, nullptr};
  int cur = 0;
  void *psi = nullptr;      // two time levels of psi, each N elements
  int pc = 0;               // which level holds psi of the current state
  void *scratch = nullptr;
  bool onepass = false;     // single-pass kernel (FP32 arithmetic forms)
  bool onepass_tma = false; // ... in its bulk-copy variant
  bool onchip = false;      // single pass with psi evaluated on chip (FP32 arithmetic, Nx even)
  bool lagged = false;      // single pass with the next psi pass one plane behind (FP32 arithmetic, Nx even)
  int *flags = nullptr;     // its per-(tile, plane) progress flags
  size_t nflags = 0;
  int stamp = 0;
  bool queued = false;      // single pass on the ordered work queue (FP32 arithmetic, D3Q19, Nx even)
  lbm::QueueState q{};      // its item table and counters (one allocation: q_mem)
  void *q_mem = nullptr;
  int q_stamp = 0;
  bool eos_f2 = false;      // EOS radicand in compensated FP32 pairs (psi pass)
  int tile = 1, zc = 0;     // its tile shape and z planes per CTA (0 = automatic)
  bool owns = false, have_buffers = false, initialized = false, psi_valid = false;
  long long steps = 0;
  int check_interval = 0;
  // profiling
  bool profiling = false;
  struct Rec { cudaEvent_t a, b; int kind; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;
  std::string err;
};

namespace {

lbm_status fail(lbm_ctx *c, lbm_status s, const std::string &msg) {
  if (c) c->err = msg;
  return s;
}

lbm_status cuda_fail(lbm_ctx *c, cudaError_t e, const char *where) {
  std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return fail(c, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, m);
}

#define CK(call, where)                                  \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
  } while (0)

// A population buffer holds Q N stored values, and at least 4N doubles: the
// spare one stages rho and u for lbm_moments (D3Q15 with FP16 storage is 30N bytes).
size_t pop_bytes(const lbm_ctx *c) {
  return std::max((size_t)c->P.q * c->P.n * lbm::storage_bytes(c->precision), (size_t)4 * c->P.n * sizeof(double));
}
size_t psi_bytes(const lbm_ctx *c) { return 2 * (size_t)c->P.n * lbm::psi_elem_bytes(c->precision); }
void *psi_at(lbm_ctx *c, int level) {
  return (char *)c->psi + (size_t)level * c->P.n * lbm::psi_elem_bytes(c->precision);
}
void *cur_psi(lbm_ctx *c) { return psi_at(c, c->pc); }

// z planes per CTA of the single-pass kernel: about eight CTAs per SM in total,
// at least 8 planes so that the two recomputed boundary planes stay cheap.
int auto_zc(const lbm_ctx *c) {
  const int bx = c->tile == lbm::kTile64x4 ? 64 : 32, by = c->tile == lbm::kTile32x8 ? 8 : 4;
  const long long tiles = (long long)((c->P.nx + bx - 1) / bx) * ((c->P.ny + by - 1) / by);
  long long chunks = (8LL * 152 + tiles / 2) / tiles;
  if (chunks < 1) chunks = 1;
  int zc = (int)((c->P.nz + chunks - 1) / chunks);
  if (zc < 8) zc = 8;
  return zc > c->P.nz ? c->P.nz : zc;
}

unsigned *err_word(lbm_ctx *c) { return (unsigned *)((char *)c->scratch + lbm::kScratchErrOffset); }
double *partials(lbm_ctx *c) { return (double *)((char *)c->scratch + lbm::kScratchPartialOffset); }
double *result(lbm_ctx *c) { return (double *)((char *)c->scratch + lbm::kScratchResultOffset); }
void *spare(lbm_ctx *c) { return c->g[c->cur ^ 1]; }

lbm_status ensure_buffers(lbm_ctx *c) {
  if (c->have_buffers) return LBM_OK;
  void *p[4] = {nullptr, nullptr, nullptr, nullptr};
  const size_t sz[4] = {pop_bytes(c), pop_bytes(c), psi_bytes(c), lbm::kScratchBytes};
  for (int k = 0; k < 4; ++k) {
    cudaError_t e = cudaMalloc(&p[k], sz[k]);
    if (e != cudaSuccess) {
      for (int j = 0; j < k; ++j) cudaFree(p[j]);
      cudaGetLastError();
      return cuda_fail(c, e, "cudaMalloc");
    }
  }
  c->g[0] = p[0];
  c->g[1] = p[1];
  c->psi = p[2];
  c->scratch = p[3];
  c->owns = true;
  c->have_buffers = true;
  CK(cudaMemsetAsync(c->scratch, 0, lbm::kScratchBytes, c->L.stream), "cudaMemsetAsync(scratch)");
  return LBM_OK;
}

cudaEvent_t pooled_event(lbm_ctx *c) {
  if (c->pool_used == c->pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c->pool.push_back(e);
  }
  return c->pool[c->pool_used++];
}

// NVTX name of a launch of the given kind (0: psi pass, 1: the step's other kernel).
const char *launch_name(const lbm_ctx *c, int kind) {
  if (kind == 0) return "lbm psi pass";
  if (c->queued) return "lbm work-list step";
  if (c->lagged) return "lbm trailing-psi single pass";
  if (c->onchip) return "lbm on-chip-psi single pass";
  if (c->onepass) return c->onepass_tma ? "lbm single pass (bulk copies)" : "lbm single pass";
  return "lbm fused pass";
}

// Launch one kernel inside an NVTX range named for it, bracketed by events
// while profiling is on.
template <typename F>
cudaError_t timed(lbm_ctx *c, int kind, F &&launch) {
  const lbm::NvtxRange range(launch_name(c, kind));
  if (!c->profiling) return launch();
  cudaEvent_t a = pooled_event(c), b = pooled_event(c);
  if (!a || !b) return cudaErrorMemoryAllocation;
  cudaEventRecord(a, c->L.stream);
  cudaError_t e = launch();
  cudaEventRecord(b, c->L.stream);
  c->recs.push_back({a, b, kind});
  return e;
}

void free_queue(lbm_ctx *c) {
  if (c->q_mem) cudaFree(c->q_mem);
  c->q_mem = nullptr;
  c->q = lbm::QueueState{};
  c->q_stamp = 0;
}

// Item table and counters of the work-list single pass (zeroed counters).
lbm_status ensure_queue(lbm_ctx *c) {
  if (c->q_mem) return LBM_OK;
  int grid = 0;
  CK(lbm::queue_grid(c->precision, &grid), "work list occupancy");
  std::vector<int4> items;
  if (!lbm::queue_items(c->P, grid, items)) return fail(c, LBM_ERR_ARG, "no valid work list for this box");
  const size_t ib = (items.size() * sizeof(int4) + 255) / 256 * 256;
  const size_t db = lbm::queue_counters(c->P) * sizeof(int);
  void *m = nullptr;
  CK(cudaMalloc(&m, ib + db), "cudaMalloc(work list)");
  c->q_mem = m;
  c->q.items = (const int4 *)m;
  c->q.nitems = (int)items.size();
  c->q.grid = grid;
  c->q.done = (int *)((char *)m + ib);
  c->q_stamp = 0;
  CK(cudaMemcpyAsync(m, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice, c->L.stream),
     "H2D work list");
  CK(cudaMemsetAsync((char *)m + ib, 0, db, c->L.stream), "clear work list counters");
  CK(cudaStreamSynchronize(c->L.stream), "cudaStreamSynchronize");  // the host table goes out of scope
  return LBM_OK;
}

lbm_status refresh_psi(lbm_ctx *c) {
  if (c->psi_valid) return LBM_OK;
  CK(lbm::launch_psi(c->P, c->precision, c->g[c->cur], cur_psi(c), err_word(c), c->L, c->eos_f2), "psi kernel");
  c->psi_valid = true;
  return LBM_OK;
}

lbm_status finish_init(lbm_ctx *c, const double *rho_dev) {
  CK(lbm::launch_state_from_rho(c->P, c->precision, rho_dev, c->g[c->cur], c->L), "state_from_rho kernel");
  c->initialized = true;
  c->psi_valid = false;
  c->steps = 0;
  return LBM_OK;
}

bool finite_positive(double v) { return std::isfinite(v) && v > 0; }

}  // namespace

extern "C" {

const char *lbm_status_string(int s) {
  switch (s) {
    case LBM_OK: return "LBM_OK";
    case LBM_ERR_ARG: return "LBM_ERR_ARG";
    case LBM_ERR_OOM: return "LBM_ERR_OOM";
    case LBM_ERR_CUDA: return "LBM_ERR_CUDA";
    case LBM_ERR_NONFINITE: return "LBM_ERR_NONFINITE";
    case LBM_ERR_EOS_DOMAIN: return "LBM_ERR_EOS_DOMAIN";
    case LBM_ERR_TIMEOUT: return "LBM_ERR_TIMEOUT";
    case LBM_ERR_STATE: return "LBM_ERR_STATE";
    case LBM_ERR_BOUNDS: return "LBM_ERR_BOUNDS";
    default: return "LBM_ERR_UNKNOWN";
  }
}

const char *lbm_last_error(const lbm_ctx *c) { return c ? c->err.c_str() : ""; }

lbm_status lbm_create(const int grid[3], const lbm_eos *eos, double G, const lbm_rates *rates, int op,
                      int precision, double sigma, void *cuda_stream, lbm_ctx **out) {
  if (!out) return LBM_ERR_ARG;
  *out = nullptr;
  KParams P;
  if (!lbm::fill_params(grid, eos, G, rates, op, precision, sigma, &P)) return LBM_ERR_ARG;
  lbm_ctx *c = new (std::nothrow) lbm_ctx();
  if (!c) return LBM_ERR_OOM;
  c->P = P;
  c->precision = precision;
  c->op = op;
  c->sigma_on = sigma != 0.0;
  c->L.stream = (cudaStream_t)cuda_stream;
  c->L.bx = 32;
  c->L.by = 4;
  // the default step: the work-list single pass where it applies and is the
  // faster one on GB300 (FP32 storage: it moves 160 instead of 236 bytes per
  // node and overlaps the FP64 EOS with the population stream), else the
  // two-pass step (FP64: bound by the FP64 pipe either way; FP16 storage: the
  // fused pass is issue-bound, and the two launches are faster)
  c->queued = lbm::queue_supported(c->P, precision) && precision == LBM_F32;
  *out = c;
  return LBM_OK;
}

lbm_status lbm_buffer_bytes(const lbm_ctx *c, size_t *pb, size_t *sb, size_t *xb) {
  if (!c) return LBM_ERR_ARG;
  if (pb) *pb = pop_bytes(c);
  if (sb) *sb = psi_bytes(c);
  if (xb) *xb = lbm::kScratchBytes;
  return LBM_OK;
}

lbm_status lbm_bind(lbm_ctx *c, void *fa, void *fb, void *psi, void *scratch) {
  if (!c) return LBM_ERR_ARG;
  if (c->have_buffers) return fail(c, LBM_ERR_STATE, "buffers already bound or allocated");
  if (!fa || !fb || !psi || !scratch || fa == fb) return fail(c, LBM_ERR_ARG, "null or aliased buffer");
  for (void *p : {fa, fb, psi, scratch})
    if (((uintptr_t)p & 255u) != 0) return fail(c, LBM_ERR_ARG, "buffers must be 256-byte aligned");
  c->g[0] = fa;
  c->g[1] = fb;
  c->psi = psi;
  c->scratch = scratch;
  c->owns = false;
  c->have_buffers = true;
  CK(cudaMemsetAsync(c->scratch, 0, lbm::kScratchBytes, c->L.stream), "cudaMemsetAsync(scratch)");
  return LBM_OK;
}

lbm_status lbm_init_droplets(lbm_ctx *c, int n, const double *centres, const double *radii, double W,
                             double rho_l, double rho_v) {
  if (!c || n < 1 || !centres || !radii) return fail(c, LBM_ERR_ARG, "bad droplet list");
  if (!finite_positive(W) || !finite_positive(rho_l) || !finite_positive(rho_v))
    return fail(c, LBM_ERR_ARG, "W, rho_l and rho_v must be positive");
  for (int k = 0; k < n; ++k)
    if (!std::isfinite(centres[3 * k]) || !std::isfinite(centres[3 * k + 1]) ||
        !std::isfinite(centres[3 * k + 2]) || !(radii[k] >= 0.0))
      return fail(c, LBM_ERR_ARG, "bad droplet centre or radius");
  lbm_status s = ensure_buffers(c);
  if (s != LBM_OK) return s;
  c->P.rho_ref = rho_v;
  lbm::refresh_float_params(c->P);
  double *rho = (double *)spare(c);
  for (int k0 = 0; k0 < n; k0 += lbm::kDropletChunk) {
    lbm::DropletChunk ch{};
    ch.count = std::min(lbm::kDropletChunk, n - k0);
    for (int k = 0; k < ch.count; ++k) {
      ch.cx[k] = centres[3 * (k0 + k)];
      ch.cy[k] = centres[3 * (k0 + k) + 1];
      ch.cz[k] = centres[3 * (k0 + k) + 2];
      ch.r[k] = radii[k0 + k];
    }
    CK(lbm::launch_rho_droplets(c->P, rho, ch, W, rho_l, rho_v, k0 == 0, c->L), "rho_droplets kernel");
  }
  return finish_init(c, rho);
}

lbm_status lbm_init_droplet(lbm_ctx *c, const double centre[3], double R, double W, double rho_l,
                            double rho_v) {
  if (!c || !centre) return fail(c, LBM_ERR_ARG, "null argument");
  return lbm_init_droplets(c, 1, centre, &R, W, rho_l, rho_v);
}

lbm_status lbm_init_flat(lbm_ctx *c, int axis, double lo, double hi, double W, double rho_l, double rho_v) {
  if (!c || axis < 0 || axis > 2 || !(lo < hi) || !std::isfinite(lo) || !std::isfinite(hi))
    return fail(c, LBM_ERR_ARG, "bad slab geometry");
  if (!finite_positive(W) || !finite_positive(rho_l) || !finite_positive(rho_v))
    return fail(c, LBM_ERR_ARG, "W, rho_l and rho_v must be positive");
  lbm_status s = ensure_buffers(c);
  if (s != LBM_OK) return s;
  c->P.rho_ref = rho_v;
  lbm::refresh_float_params(c->P);
  double *rho = (double *)spare(c);
  CK(lbm::launch_rho_slab(c->P, rho, axis, lo, hi, W, rho_l, rho_v, c->L), "rho_slab kernel");
  return finish_init(c, rho);
}

lbm_status lbm_init_field(lbm_ctx *c, const double *rho, int on_device, double rho_ref) {
  if (!c || !rho || !std::isfinite(rho_ref)) return fail(c, LBM_ERR_ARG, "null field or bad rho_ref");
  lbm_status s = ensure_buffers(c);
  if (s != LBM_OK) return s;
  c->P.rho_ref = rho_ref;
  lbm::refresh_float_params(c->P);
  const double *src = rho;
  if (!on_device) {
    double *tmp = (double *)spare(c);
    CK(cudaMemcpyAsync(tmp, rho, sizeof(double) * c->P.n, cudaMemcpyHostToDevice, c->L.stream),
       "cudaMemcpyAsync(rho H2D)");
    src = tmp;
  }
  s = finish_init(c, src);
  if (s != LBM_OK) return s;
  if (!on_device) CK(cudaStreamSynchronize(c->L.stream), "cudaStreamSynchronize");
  return LBM_OK;
}

lbm_status lbm_check(lbm_ctx *c) {
  if (!c) return LBM_ERR_ARG;
  if (!c->have_buffers) return LBM_OK;
  unsigned w = 0;
  CK(cudaMemcpyAsync(&w, err_word(c), sizeof(unsigned), cudaMemcpyDeviceToHost, c->L.stream), "read error word");
  CK(cudaMemsetAsync(err_word(c), 0, sizeof(unsigned), c->L.stream), "clear error word");
  CK(cudaStreamSynchronize(c->L.stream), "cudaStreamSynchronize");
  if (lbm::dbg::take_all()) return fail(c, LBM_ERR_BOUNDS, "a kernel index fell outside its buffer (debug build)");
  if (w & lbm::kErrTimeout)
    return fail(c, LBM_ERR_TIMEOUT, "a bounded wait gave up, or a work-list launch could not follow its list");
  if (w & lbm::kErrNonFinite) return fail(c, LBM_ERR_NONFINITE, "non-finite density");
  if (w & lbm::kErrEosDomain) return fail(c, LBM_ERR_EOS_DOMAIN, "density left the domain of the EOS");
  return LBM_OK;
}

lbm_status lbm_step(lbm_ctx *c, int n) {
  if (!c) return LBM_ERR_ARG;
  if (n < 1) return fail(c, LBM_ERR_ARG, "n must be >= 1");
  if (!c->initialized) return fail(c, LBM_ERR_STATE, "lbm_step before an init");
  if (c->queued) {
    lbm_status s = ensure_queue(c);
    if (s != LBM_OK) return s;
  }
  if ((c->onepass || c->lagged || c->queued) && !c->psi_valid) {
    CK(timed(c, 0, [&] {
         return lbm::launch_psi(c->P, c->precision, c->g[c->cur], cur_psi(c), err_word(c), c->L,
                                (c->lagged || c->queued) && c->eos_f2);
       }),
       "psi kernel");
    c->psi_valid = true;
  }
  const int zc = c->zc > 0 ? c->zc : auto_zc(c);
  for (int k = 0; k < n; ++k) {
    void *gin = c->g[c->cur], *gout = c->g[c->cur ^ 1];
    if (c->queued) {
      void *pin = cur_psi(c), *pout = psi_at(c, c->pc ^ 1);
      // the counters advance only with launches that run (each one claims every item once)
      const int stamp = c->q_stamp + 1;
      CK(timed(c, 1, [&] {
           return lbm::launch_queue(c->P, c->precision, c->op, c->sigma_on, c->eos_f2, gin, gout, pin, pout, c->q,
                                    stamp, err_word(c), c->L.stream);
         }),
         "single-pass kernel");
      c->q_stamp = stamp;
      c->pc ^= 1;
      c->cur ^= 1;
      c->psi_valid = true;
    } else if (c->lagged) {
      void *pin = cur_psi(c), *pout = psi_at(c, c->pc ^ 1);
      const int stamp = ++c->stamp;
      CK(timed(c, 1, [&] {
           return lbm::launch_lagged(c->P, c->precision, c->op, c->sigma_on, c->eos_f2, gin, gout, pin, pout,
                                     c->flags, stamp, err_word(c), c->L.stream);
         }),
         "single-pass kernel");
      c->pc ^= 1;
      c->cur ^= 1;
      c->psi_valid = true;
    } else if (c->onchip) {
      CK(timed(c, 1, [&] {
           return lbm::launch_onchip(c->P, c->precision, c->op, c->sigma_on, c->eos_f2, gin, gout, err_word(c),
                                     c->L.stream);
         }),
         "single-pass kernel");
      c->cur ^= 1;
      c->psi_valid = false;
    } else if (c->onepass) {
      void *pin = cur_psi(c), *pout = psi_at(c, c->pc ^ 1);
      CK(timed(c, 1, [&] {
           return c->onepass_tma ? lbm::launch_onepass_tma(c->P, c->precision, c->op, c->sigma_on, zc, gin, gout,
                                                           pin, pout, err_word(c), c->L.stream)
                                 : lbm::launch_onepass(c->P, c->precision, c->op, c->sigma_on, c->tile, zc, gin,
                                                       gout, pin, pout, err_word(c), c->L.stream);
         }),
         "single-pass kernel");
      c->pc ^= 1;
      c->cur ^= 1;
      c->psi_valid = true;
    } else {
      void *psi = cur_psi(c);
      CK(timed(c, 0, [&] { return lbm::launch_psi(c->P, c->precision, gin, psi, err_word(c), c->L, c->eos_f2); }),
         "psi kernel");
      CK(timed(c, 1, [&] {
           return lbm::launch_fused(c->P, c->precision, c->op, c->sigma_on, gin, gout, psi, c->L);
         }),
         "fused kernel");
      c->cur ^= 1;
      c->psi_valid = false;
    }
    ++c->steps;
    if (c->check_interval > 0 && c->steps % c->check_interval == 0) {
      lbm_status s = lbm_check(c);
      if (s != LBM_OK) return s;
    }
  }
  return LBM_OK;
}

lbm_status lbm_moments(lbm_ctx *c, double *rho, double *u, int on_device) {
  if (!c || (!rho && !u)) return fail(c, LBM_ERR_ARG, "no output");
  if (!c->initialized) return fail(c, LBM_ERR_STATE, "no state");
  lbm_status s = refresh_psi(c);
  if (s != LBM_OK) return s;
  const size_t n = c->P.n;
  if (on_device) {
    CK(lbm::launch_moments(c->P, c->precision, c->g[c->cur], cur_psi(c), rho, u, c->L), "moments kernel");
    return LBM_OK;
  }
  double *tmp = (double *)spare(c);  // 4N doubles fit in any population buffer
  CK(lbm::launch_moments(c->P, c->precision, c->g[c->cur], cur_psi(c), tmp, tmp + n, c->L), "moments kernel");
  if (rho) CK(cudaMemcpyAsync(rho, tmp, sizeof(double) * n, cudaMemcpyDeviceToHost, c->L.stream), "D2H rho");
  if (u) CK(cudaMemcpyAsync(u, tmp + n, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c->L.stream), "D2H u");
  CK(cudaStreamSynchronize(c->L.stream), "cudaStreamSynchronize");
  return LBM_OK;
}

lbm_status lbm_get_populations(lbm_ctx *c, double *f, int on_device) {
  if (!c || !f) return fail(c, LBM_ERR_ARG, "null output");
  if (!c->initialized) return fail(c, LBM_ERR_STATE, "no state");
  const size_t n = c->P.n;
  if (on_device) {
    CK(lbm::launch_get_populations(c->P, c->precision, c->g[c->cur], f, 0, c->P.q, c->L), "get_populations kernel");
    return LBM_OK;
  }
  double *tmp = (double *)spare(c);
  for (int a = 0; a < c->P.q; ++a) {
    CK(lbm::launch_get_populations(c->P, c->precision, c->g[c->cur], tmp, a, a + 1, c->L),
       "get_populations kernel");
    CK(cudaMemcpyAsync(f + a * n, tmp, sizeof(double) * n, cudaMemcpyDeviceToHost, c->L.stream), "D2H f");
    CK(cudaStreamSynchronize(c->L.stream), "cudaStreamSynchronize");
  }
  return LBM_OK;
}

lbm_status lbm_set_populations(lbm_ctx *c, const double *f, int on_device) {
  if (!c || !f) return fail(c, LBM_ERR_ARG, "null input");
  if (!c->initialized) return fail(c, LBM_ERR_STATE, "set_populations needs an init (for rho_ref)");
  const size_t n = c->P.n;
  if (on_device) {
    CK(lbm::launch_set_populations(c->P, c->precision, f, c->g[c->cur], 0, c->P.q, c->L), "set_populations kernel");
  } else {
    double *tmp = (double *)spare(c);
    for (int a = 0; a < c->P.q; ++a) {
      CK(cudaMemcpyAsync(tmp, f + a * n, sizeof(double) * n, cudaMemcpyHostToDevice, c->L.stream), "H2D f");
      CK(lbm::launch_set_populations(c->P, c->precision, tmp, c->g[c->cur], a, a + 1, c->L),
         "set_populations kernel");
      CK(cudaStreamSynchronize(c->L.stream), "cudaStreamSynchronize");
    }
  }
  c->psi_valid = false;
  c->steps = 0;
  return LBM_OK;
}

lbm_status lbm_diag(lbm_ctx *c, double out[5]) {
  if (!c || !out) return fail(c, LBM_ERR_ARG, "null output");
  if (!c->initialized) return fail(c, LBM_ERR_STATE, "no state");
  lbm_status s = refresh_psi(c);
  if (s != LBM_OK) return s;
  CK(lbm::launch_diag(c->P, c->precision, c->g[c->cur], cur_psi(c), partials(c), result(c), c->L), "diag kernels");
  CK(cudaMemcpyAsync(out, result(c), 5 * sizeof(double), cudaMemcpyDeviceToHost, c->L.stream), "D2H diag");
  CK(cudaStreamSynchronize(c->L.stream), "cudaStreamSynchronize");
  return LBM_OK;
}

lbm_status lbm_set_check_interval(lbm_ctx *c, int k) {
  if (!c || k < 0) return LBM_ERR_ARG;
  c->check_interval = k;
  return LBM_OK;
}

lbm_status lbm_set_profiling(lbm_ctx *c, int enabled) {
  if (!c) return LBM_ERR_ARG;
  c->profiling = enabled != 0;
  return LBM_OK;
}

lbm_status lbm_kernel_times(lbm_ctx *c, double *ms_psi, long long *n_psi, double *ms_fused, long long *n_fused) {
  if (!c) return LBM_ERR_ARG;
  CK(cudaStreamSynchronize(c->L.stream), "cudaStreamSynchronize");
  double t[2] = {0, 0};
  long long cnt[2] = {0, 0};
  for (auto &r : c->recs) {
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, r.a, r.b), "cudaEventElapsedTime");
    t[r.kind] += ms;
    cnt[r.kind] += 1;
  }
  c->recs.clear();
  c->pool_used = 0;
  if (ms_psi) *ms_psi = t[0];
  if (n_psi) *n_psi = cnt[0];
  if (ms_fused) *ms_fused = t[1];
  if (n_fused) *n_fused = cnt[1];
  return LBM_OK;
}

lbm_status lbm_set_tuning(lbm_ctx *c, int single_pass, int tile, int z_planes) {
  if (!c || single_pass < 0 || single_pass > 5 || tile < 0 || tile > 2 || z_planes < 0)
    return fail(c, LBM_ERR_ARG, "bad tuning");
  if (single_pass && c->precision == LBM_F64) return fail(c, LBM_ERR_ARG, "single pass needs FP32 arithmetic");
  if (single_pass && single_pass != 5 && c->P.q == 15)
    return fail(c, LBM_ERR_ARG, "the single-pass variants other than the work list are D3Q19 kernels");
  if (single_pass == 2 && !lbm::onepass_tma_supported(c->P, c->precision))
    return fail(c, LBM_ERR_ARG, "bulk-copy single pass needs FP32 storage, Nx % 4 == 0 and Nx >= 40");
  if (single_pass == 3 && !lbm::onchip_supported(c->P, c->precision))
    return fail(c, LBM_ERR_ARG, "on-chip-psi single pass needs FP32 arithmetic and an even Nx");
  if (single_pass == 5 && !lbm::queue_supported(c->P, c->precision))
    return fail(c, LBM_ERR_ARG, "work-queue single pass needs FP32 arithmetic and an even Nx");
  if (single_pass == 4) {
    if (!lbm::lagged_supported(c->P, c->precision))
      return fail(c, LBM_ERR_ARG, "trailing-psi single pass needs FP32 arithmetic and an even Nx");
    const size_t need = lbm::lagged_flag_count(c->P);
    if (c->nflags < need) {
      if (c->flags) cudaFree(c->flags);
      c->flags = nullptr;
      c->nflags = 0;
      CK(cudaMalloc((void **)&c->flags, need * sizeof(int)), "cudaMalloc(flags)");
      CK(cudaMemsetAsync(c->flags, 0, need * sizeof(int), c->L.stream), "cudaMemsetAsync(flags)");
      c->nflags = need;
      c->stamp = 0;
    }
  }
  c->psi_valid = false;
  c->queued = single_pass == 5;
  c->lagged = single_pass == 4;
  c->onchip = single_pass == 3;
  c->onepass = single_pass == 1 || single_pass == 2;
  c->onepass_tma = single_pass == 2;
  if (c->onepass_tma) tile = lbm::kTile32x8;
  c->tile = tile;
  c->zc = z_planes;
  return LBM_OK;
}

lbm_status lbm_set_variable_viscosity(lbm_ctx *c, double rho_l, double rho_v, double nu_l, double nu_v) {
  if (!c) return LBM_ERR_ARG;
  if (nu_l <= 0.0 && nu_v <= 0.0) {
    c->P.varnu = 0;
    return LBM_OK;
  }
  if (!(std::isfinite(rho_l) && std::isfinite(rho_v) && rho_l != rho_v && nu_l > 0.0 && nu_v > 0.0))
    return fail(c, LBM_ERR_ARG, "need rho_l != rho_v and positive nu_l, nu_v");
  c->P.varnu = 1;
  c->P.nu_v = nu_v;
  c->P.rho_v_nu = rho_v;
  c->P.nu_slope = (nu_l - nu_v) / (rho_l - rho_v);
  c->P.nu_lo = std::min(nu_l, nu_v);
  c->P.nu_hi = std::max(nu_l, nu_v);
  lbm::refresh_float_params(c->P);
  return LBM_OK;
}

lbm_status lbm_set_eos_arith(lbm_ctx *c, int mode) {
  if (!c || mode < 0 || mode > 1) return fail(c, LBM_ERR_ARG, "bad EOS arithmetic mode");
  if (mode == 1 && c->precision == LBM_F64) return fail(c, LBM_ERR_ARG, "the FP64 form evaluates its EOS in FP64");
  c->eos_f2 = mode == 1;
  c->psi_valid = false;
  return LBM_OK;
}

lbm_status lbm_set_wait_budget(lbm_ctx *c, int spin_limit, int inject_unreachable) {
  if (!c) return LBM_ERR_ARG;
  c->P.spin_limit = spin_limit > 0 ? spin_limit : lbm::kDefaultSpinLimit;
  c->P.wait_bias = inject_unreachable ? 1 : 0;
  return LBM_OK;
}

lbm_status lbm_get_tuning(const lbm_ctx *c, int *single_pass, int *tile, int *z_planes) {
  if (!c) return LBM_ERR_ARG;
  if (single_pass)
    *single_pass = c->queued ? 5 : c->lagged ? 4 : c->onchip ? 3 : c->onepass ? (c->onepass_tma ? 2 : 1) : 0;
  if (tile) *tile = c->tile;
  if (z_planes) *z_planes = c->zc > 0 ? c->zc : auto_zc(c);
  return LBM_OK;
}

long long lbm_step_count(const lbm_ctx *c) { return c ? c->steps : -1; }

void lbm_destroy(lbm_ctx *c) {
  if (!c) return;
  if (c->have_buffers || !c->pool.empty() || c->flags || c->q_mem) cudaStreamSynchronize(c->L.stream);
  for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
  if (c->flags) cudaFree(c->flags);
  free_queue(c);
  if (c->owns) {
    cudaFree(c->g[0]);
    cudaFree(c->g[1]);
    cudaFree(c->psi);
    cudaFree(c->scratch);
  }
  delete c;
}

}  // extern "C"

// Registry of the debug build's per-translation-unit bounds-error readers
// (empty in the normal build).
namespace lbm {
namespace dbg {
static std::vector<unsigned (*)()> &readers() {
  static std::vector<unsigned (*)()> r;
  return r;
}
bool register_reader(unsigned (*r)()) {
  readers().push_back(r);
  return true;
}
unsigned take_all() {
  unsigned v = 0;
  for (auto r : readers()) v |= r();
  return v;
}
}  // namespace dbg
}  // namespace lbm

// Read-only view of a context's parameters for other translation units.
namespace lbm {
bool ctx_params(const lbm_ctx *c, KParams *P, int *precision, int *op, bool *sigma_on, cudaStream_t *stream) {
  if (!c) return false;
  *P = c->P;
  *precision = c->precision;
  *op = c->op;
  *sigma_on = c->sigma_on;
  *stream = c->L.stream;
  return true;
}
}  // namespace lbm

// Validate a box description and fill the kernel parameters (shared by
// lbm_create and lbm_batch_add).
namespace lbm {
bool fill_params(const int grid[3], const lbm_eos *eos, double G, const lbm_rates *rates, int op, int precision,
                 double sigma, KParams *out) {
  if (!grid || !eos || !rates || !out) return false;
  if (grid[0] < 3 || grid[1] < 3 || grid[2] < 3) return false;
  const long long n = (long long)grid[0] * grid[1] * grid[2];
  // 32-bit node index, unsigned 32-bit element offsets (19 N < 2^32), grid.z limit
  if (n >= (1LL << 31) || 19 * n >= (1LL << 32) || grid[2] > 65535) return false;
  if (op != LBM_OP_ORTHOGONAL && op != LBM_OP_NONORTHOGONAL && op != LBM_OP_NONORTHOGONAL_D3Q15) return false;
  if (precision < LBM_F64 || precision > LBM_F32_STORE_F16) return false;
  if (eos->kind < LBM_EOS_CS || eos->kind > LBM_EOS_NONE) return false;
  const double rs[6] = {rates->s_e, rates->s_nu, rates->s_q, rates->s_pi, rates->s_eps, rates->s_m};
  for (double s : rs)
    if (!(s > 0.0 && s < 2.0)) return false;  // stable range of a relaxation rate
  if (!std::isfinite(G) || !std::isfinite(sigma)) return false;
  if (eos->kind == LBM_EOS_CS) {
    if (!finite_positive(eos->b) || !finite_positive(eos->R) || !finite_positive(eos->T) || !std::isfinite(eos->a) ||
        G == 0.0)
      return false;
  } else if (eos->kind == LBM_EOS_EXP) {
    if (!std::isfinite(eos->psi0) || !finite_positive(eos->rho0)) return false;
  }
  if (sigma != 0.0 && eos->kind == LBM_EOS_NONE) return false;
  KParams P{};
  P.nx = grid[0];
  P.ny = grid[1];
  P.nz = grid[2];
  P.n = (int)n;
  P.q = op == LBM_OP_NONORTHOGONAL_D3Q15 ? 15 : 19;
  P.G = eos->kind == LBM_EOS_NONE ? 0.0 : G;
  P.rho_ref = 0.0;
  P.s_e = rates->s_e;
  P.s_nu = rates->s_nu;
  P.s_q = rates->s_q;
  P.s_pi = rates->s_pi;
  P.s_eps = rates->s_eps;
  P.s_m = rates->s_m;
  P.sigma_coef = 6.0 * sigma * G * G / (1.0 / rates->s_e - 0.5);
  P.eos = eos->kind;
  P.a = eos->a;
  P.b = eos->b;
  P.RT = eos->R * eos->T;
  P.psi0 = eos->psi0;
  P.rho0 = eos->rho0;
  P.b4 = 0.25 * eos->b;
  P.two_over_G = P.G != 0.0 ? 2.0 / P.G : 0.0;
  {
    // coefficients of the radicand polynomial (see KParams)
    const double cc = P.b4, rt = P.RT, aa = P.a, k = P.two_over_G;
    P.q0 = k * (rt - 1.0 / 3.0);
    P.q1 = k * (rt * cc - aa + cc);
    P.q2 = k * (rt * cc * cc + 3.0 * aa * cc - cc * cc);
    P.q3 = k * (-rt * cc * cc * cc - 3.0 * aa * cc * cc + cc * cc * cc / 3.0);
    P.q4 = k * (aa * cc * cc * cc);
    P.f_rho_max = eos->b > 0 ? (float)(4.0 / eos->b) : 0.0f;
  }
  P.spin_limit = kDefaultSpinLimit;
  P.wait_bias = 0;
  refresh_float_params(P);
  *out = P;
  return true;
}
}  // namespace lbm
