// Batched boxes: many independent periodic boxes advanced together, the
// launches of two steps captured in a CUDA graph.  Boxes with an even Nx step
// on the work list (one cooperative launch) or on the two-pass pair kernels
// (the fused pass as a flat grid per operator, then psi of the new level over
// work items); boxes with an odd Nx on the one-node single pass, in the same
// step graph.  Boxes can join and leave
// between calls (continuous batching); each box's buffers come from the
// stream-ordered allocator and count against the batch's HBM budget.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_device.cuh"
#include "lbm_internal.h"

using lbm::BatchBox;
using lbm::KParams;

namespace lbm {
bool fill_params(const int grid[3], const lbm_eos *eos, double G, const lbm_rates *rates, int op, int precision,
                 double sigma, KParams *P);
}

namespace {

// lbm_batch_set_tuning's tile value for the work-list single pass (64x4 tile jobs)
constexpr int kTileWorkList = 3;

struct HostBox {
  bool live = false;
  BatchBox d{};        // descriptor as the kernel sees it
  int precision = 0;
  bool initialised = false;
  int zc = 0;          // planes per work item
  size_t bytes = 0;    // device bytes held
  void *mem = nullptr; // one allocation: g0, g1, psi0, psi1, u_prev
  float *u_prev = nullptr;
  long long steps = 0;
};

}  // namespace

struct lbm_batch {
  int precision = 1, eos = 0;
  cudaStream_t stream = nullptr;
  size_t budget = 0, used = 0;
  int tile = kTileWorkList;  // step kind: the work list, or the tile shape of the other kernels
  int grid_blocks = 0;       // SMs (persistent grid sizes are multiples of it)
  std::vector<HostBox> boxes;
  BatchBox *d_boxes = nullptr;
  int4 *d_items = nullptr;
  int cap_boxes = 0, cap_items = 0, nitems = 0;
  unsigned *d_err = nullptr;
  void *d_scratch = nullptr; // reduction partials of lbm_batch_diag
  double *d_red = nullptr;   // per-box reduction results (max |du|)
  bool own_stream = false;
  int cap_red = 0;
  bool dirty = true;         // descriptors / items need uploading, graphs re-capturing
  bool pair = false;         // the captured step is the two-pass pair kernels
  bool wl = false;           // ... or the work-list single pass
  bool odd = false;          // ... and the one-node single pass for the odd-Nx boxes
  int *d_done = nullptr;     // its completion counters, cleared before every launch
  int *d_fmap = nullptr;     // two-pass step: the box of every block of the flat fused grids
  long long cap_fmap = 0;
  int fused_blocks[2] = {0, 0};  // ... non-orthogonal boxes' blocks, then orthogonal
  long long cap_done = 0, ndone = 0;
  int wl_grid = 0;
  // graphs of two steps and of one step, for each starting parity: the state of
  // box h is at level h.d.cur ^ phase, and a step at parity `phase` moves it to
  // the other level, so an odd step count flips phase instead of the descriptors
  cudaGraphExec_t g2[2] = {nullptr, nullptr}, g1[2] = {nullptr, nullptr};
  int phase = 0;
  long long builds = 0;      // descriptor uploads and graph captures so far
  long long steps = 0;
  std::string err;
};

namespace {

lbm_status bfail(lbm_batch *b, lbm_status s, const std::string &m) {
  if (b) b->err = m;
  return s;
}

#define BCK(call, where)                                                                         \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      return bfail(b, e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,               \
                   std::string(where) + ": " + cudaGetErrorString(e_));                          \
  } while (0)

size_t box_bytes(int precision, long long n) {
  const size_t pop = (size_t)19 * n * lbm::storage_bytes(precision);
  auto up = [](size_t v) { return (v + 255) / 256 * 256; };
  return 2 * up(pop) + 2 * up((size_t)n * 4) + up((size_t)3 * n * 4);
}

// Ints after a work list's completion counters for the blocks' item-claim counter (at offset 16).
constexpr long long kClaimInts = 32;

// Planes per work item unless tuned: 32 (two of them are recomputed).
int default_zc(const KParams &P) { return std::min(P.nz, 32); }

void destroy_graphs(lbm_batch *b) {
  for (int p = 0; p < 2; ++p) {
    if (b->g2[p]) cudaGraphExecDestroy(b->g2[p]);
    if (b->g1[p]) cudaGraphExecDestroy(b->g1[p]);
    b->g2[p] = b->g1[p] = nullptr;
  }
}

// Upload descriptors and the work-item table (largest boxes first), recapture graphs.
lbm_status rebuild(lbm_batch *b) {
  // fold the phase into the descriptors: afterwards level d.cur holds each state
  for (auto &h : b->boxes)
    if (h.live) h.d.cur ^= b->phase;
  b->phase = 0;
  const int nb = (int)b->boxes.size();
  if (nb > b->cap_boxes) {
    if (b->d_boxes) cudaFreeAsync(b->d_boxes, b->stream);
    BCK(cudaMallocAsync((void **)&b->d_boxes, sizeof(BatchBox) * std::max(nb, 1), b->stream), "box table");
    b->cap_boxes = nb;
  }
  std::vector<BatchBox> desc(std::max(nb, 1));
  std::vector<std::pair<long long, int>> order;
  for (int i = 0; i < nb; ++i) {
    desc[i] = b->boxes[i].d;
    if (b->boxes[i].live && b->boxes[i].initialised) order.push_back({(long long)b->boxes[i].d.P.n, i});
  }
  std::sort(order.begin(), order.end(), [](auto &x, auto &y) { return x.first > y.first || (x.first == y.first && x.second < y.second); });
  // boxes with an even Nx step on the two-node kernels (the work list, or the two-pass pair kernels);
  // boxes with an odd Nx on the one-node single pass; one step graph runs both groups
  std::vector<std::pair<long long, int>> even, odd;
  for (auto &o : order) (b->boxes[o.second].d.P.nx % 2 == 0 ? even : odd).push_back(o);
  const bool wl = !even.empty() && b->tile == kTileWorkList;
  const int tile = b->tile == kTileWorkList ? lbm::kTile32x8 : b->tile;  // of the tile-shaped kernels
  std::vector<int4> items;
  auto tile_items = [&](const std::vector<std::pair<long long, int>> &group) {
    int bx, by;
    lbm::onepass_tile_shape(tile, &bx, &by);
    for (auto &o : group) {
      const HostBox &h = b->boxes[o.second];
      const KParams &P = h.d.P;
      const int tx = (P.nx + bx - 1) / bx, ty = (P.ny + by - 1) / by, zc = h.zc > 0 ? h.zc : default_zc(P);
      for (int z0 = 0; z0 < P.nz; z0 += zc)
        for (int j = 0; j < ty; ++j)
          for (int i = 0; i < tx; ++i)
            items.push_back(make_int4(o.second, i | (j << 16), z0, std::min(z0 + zc, P.nz)));
    }
  };
  if (wl) {
    // the work list over the even-Nx boxes in this order; each box's counters start at its qbase
    BCK(lbm::batch_queue_grid(b->precision, b->eos, &b->wl_grid), "work list occupancy");
    std::vector<const KParams *> ps;
    for (auto &o : even) ps.push_back(&b->boxes[o.second].d.P);
    std::vector<int> base;
    long long nc = 0;
    if (!lbm::batch_queue_items(ps, b->wl_grid, items, base, &nc)) return bfail(b, LBM_ERR_ARG, "no valid work list");
    for (size_t k = 0; k < even.size(); ++k) {
      BatchBox &d = b->boxes[even[k].second].d;
      d.qbase = base[k];
      lbm::batch_queue_geometry(d);
      desc[even[k].second] = d;
    }
    // the list numbers boxes in `even`; the kernel reads the descriptor table by slot: renumber, then
    // check every job against the descriptor it will read (plane and tile inside that box, counter
    // inside the counter array)
    for (auto &it : items) {
      if (it.x >= 0) it.x = even[it.x].second;
      if (it.z >= 0) it.z = even[it.z].second;
      for (int side = 0; side < 2; ++side) {
        const int slot = side ? it.z : it.x;
        if (slot < 0) continue;
        const KParams &P = desc[slot].P;
        const unsigned zt = (unsigned)(side ? it.w : it.y);
        const long long z = zt & 0xffffu, t = zt >> 16;
        const long long T = lbm::batch_queue_tiles(P);
        if (slot >= nb || !b->boxes[slot].live || P.nx % 2 != 0 || z >= P.nz || t >= T ||
            desc[slot].qbase + P.nz * T > nc)
          return bfail(b, LBM_ERR_ARG, "work list does not match the box table");
      }
    }
    if (nc + kClaimInts > b->cap_done) {  // the counters, then the blocks' item-claim counter
      if (b->d_done) cudaFreeAsync(b->d_done, b->stream);
      b->d_done = nullptr;
      BCK(cudaMallocAsync((void **)&b->d_done, sizeof(int) * (nc + kClaimInts), b->stream), "work list counters");
      b->cap_done = nc + kClaimInts;
    }
    b->ndone = nc;
  } else {
    tile_items(even);
    // the flat fused grids: one block per plane of a tile, non-orthogonal boxes first, box by box
    int bx, by;
    lbm::onepass_tile_shape(tile, &bx, &by);
    std::vector<int> fmap;
    for (int g = 0; g < 2; ++g) {
      const int op = g == 0 ? lbm::kNonOrth : lbm::kOrth;
      const size_t before = fmap.size();
      for (auto &o : even) {
        BatchBox &d = b->boxes[o.second].d;
        if (d.op != op) continue;
        const long long T = (long long)((d.P.nx + bx - 1) / bx) * ((d.P.ny + by - 1) / by);
        if ((long long)fmap.size() + T * d.P.nz > (1LL << 31) - 1) return bfail(b, LBM_ERR_ARG, "batch too large");
        d.qbase = (int)fmap.size();
        desc[o.second].qbase = d.qbase;
        fmap.insert(fmap.end(), (size_t)(T * d.P.nz), o.second);
      }
      b->fused_blocks[g] = (int)(fmap.size() - before);
    }
    if ((long long)fmap.size() > b->cap_fmap) {
      if (b->d_fmap) cudaFreeAsync(b->d_fmap, b->stream);
      b->d_fmap = nullptr;
      BCK(cudaMallocAsync((void **)&b->d_fmap, sizeof(int) * fmap.size(), b->stream), "fused block map");
      b->cap_fmap = (long long)fmap.size();
    }
    if (!fmap.empty())
      BCK(cudaMemcpyAsync(b->d_fmap, fmap.data(), sizeof(int) * fmap.size(), cudaMemcpyHostToDevice, b->stream),
          "H2D fused block map");
    BCK(cudaStreamSynchronize(b->stream), "sync");  // fmap goes out of scope
  }
  const int n_even = (int)items.size();
  tile_items(odd);
  if ((int)items.size() > b->cap_items) {
    if (b->d_items) cudaFreeAsync(b->d_items, b->stream);
    BCK(cudaMallocAsync((void **)&b->d_items, sizeof(int4) * items.size(), b->stream), "item table");
    b->cap_items = (int)items.size();
  }
  b->nitems = (int)items.size();
  if (nb) BCK(cudaMemcpyAsync(b->d_boxes, desc.data(), sizeof(BatchBox) * nb, cudaMemcpyHostToDevice, b->stream), "H2D boxes");
  if (b->nitems)
    BCK(cudaMemcpyAsync(b->d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, b->stream), "H2D items");
  BCK(cudaStreamSynchronize(b->stream), "sync");  // host vectors go out of scope
  destroy_graphs(b);
  b->wl = wl;
  b->pair = !wl && n_even > 0;
  b->odd = b->nitems > n_even;
  if (b->nitems) {
    // resident blocks per SM: the pair kernels' own occupancy (the psi kernel needs half the fused kernel's
    // registers), the single-pass kernel's launch bounds
    int pair_per_sm[2] = {1, 1};
    if (b->pair) BCK(lbm::batch_pair_occupancy(b->precision, b->eos, tile, pair_per_sm), "pair kernel occupancy");
    const int per_sm = tile == lbm::kTile32x4 ? 4 : 2;
    const int n_odd = b->nitems - n_even;
    const int grid_odd = std::min(b->grid_blocks * per_sm, std::max(n_odd, 1));
    auto step = [&](int parity) {
      cudaError_t e = cudaSuccess;
      if (wl) {
        e = cudaMemsetAsync(b->d_done, 0, sizeof(int) * (size_t)(b->ndone + kClaimInts), b->stream);
        if (e == cudaSuccess)
          e = lbm::launch_batch_queue(b->precision, b->eos, b->d_boxes, b->d_items, n_even, parity, b->wl_grid,
                                      b->d_done, (int)b->ndone, b->d_err, b->stream);
      } else if (n_even) {
        e = lbm::launch_batch_pair(b->precision, b->eos, tile, b->d_boxes, b->d_items, n_even, b->d_fmap,
                                   b->fused_blocks, parity, b->grid_blocks, pair_per_sm, b->d_err, b->stream);
      }
      if (e == cudaSuccess && n_odd)
        e = lbm::launch_batch_onepass(b->precision, b->eos, tile, b->d_boxes, b->d_items + n_even, n_odd, parity,
                                      grid_odd, b->d_err, b->stream);
      return e;
    };
    for (int k = 0; k < 4; ++k) {  // g2[0], g2[1], g1[0], g1[1]
      const int two = k < 2, p0 = k & 1;
      cudaGraph_t g;
      BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
      cudaError_t e = step(p0);
      if (e == cudaSuccess && two) e = step(p0 ^ 1);
      cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (e2 == cudaSuccess) cudaGraphDestroy(g);
        return bfail(b, LBM_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
      }
      cudaGraphExec_t x;
      e = cudaGraphInstantiate(&x, g, 0);
      cudaGraphDestroy(g);
      BCK(e, "graph instantiate");
      (two ? b->g2 : b->g1)[p0] = x;
    }
  }
  ++b->builds;
  b->dirty = false;
  return LBM_OK;
}

HostBox *get_box(lbm_batch *b, int id) {
  if (!b || id < 0 || id >= (int)b->boxes.size() || !b->boxes[id].live) return nullptr;
  return &b->boxes[id];
}

lbm::Launch launch_of(lbm_batch *b) {
  lbm::Launch L;
  L.stream = b->stream;
  L.bx = 32;
  L.by = 4;
  return L;
}

// Level of a box's current state (see lbm_batch::phase).
int cur_level(const lbm_batch *b, const HostBox *h) { return h->d.cur ^ b->phase; }
void *cur_g(const lbm_batch *b, HostBox *h) { return h->d.g[cur_level(b, h)]; }
float *cur_psi(const lbm_batch *b, HostBox *h) { return h->d.psi[cur_level(b, h)]; }
void *spare_g(const lbm_batch *b, HostBox *h) { return h->d.g[cur_level(b, h) ^ 1]; }

lbm_status finish_box_init(lbm_batch *b, HostBox *h, const double *rho_dev) {
  const lbm::Launch L = launch_of(b);
  BCK(lbm::launch_state_from_rho(h->d.P, h->precision, rho_dev, cur_g(b, h), L), "state_from_rho");
  BCK(lbm::launch_psi(h->d.P, h->precision, cur_g(b, h), cur_psi(b, h), b->d_err, L), "psi");
  BCK(cudaMemsetAsync(h->u_prev, 0, sizeof(float) * 3 * (size_t)h->d.P.n, b->stream), "clear u_prev");
  h->initialised = true;
  h->steps = 0;
  b->dirty = true;
  return LBM_OK;
}

}  // namespace

extern "C" {

size_t lbm_batch_box_bytes(int precision, const int grid[3]) {
  if (!grid || grid[0] < 3 || grid[1] < 3 || grid[2] < 3) return 0;
  return box_bytes(precision, (long long)grid[0] * grid[1] * grid[2]);
}

lbm_status lbm_batch_create(int precision, int eos_kind, size_t hbm_budget_bytes, void *cuda_stream,
                            lbm_batch **out) {
  if (!out) return LBM_ERR_ARG;
  *out = nullptr;
  if (precision != LBM_F32 && precision != LBM_F32_STORE_F16) return LBM_ERR_ARG;
  if (eos_kind < LBM_EOS_CS || eos_kind > LBM_EOS_NONE) return LBM_ERR_ARG;
  lbm_batch *b = new (std::nothrow) lbm_batch();
  if (!b) return LBM_ERR_OOM;
  b->precision = precision;
  b->eos = eos_kind;
  b->stream = (cudaStream_t)cuda_stream;
  b->budget = hbm_budget_bytes;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    delete b;
    return LBM_ERR_CUDA;
  }
  b->grid_blocks = sms;
  if (!b->stream) {  // graphs cannot be captured on the legacy default stream
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return LBM_ERR_CUDA;
    }
    b->own_stream = true;
  }
  if (cudaMallocAsync((void **)&b->d_err, 256, b->stream) != cudaSuccess ||
      cudaMemsetAsync(b->d_err, 0, 256, b->stream) != cudaSuccess ||
      cudaMallocAsync(&b->d_scratch, lbm::kScratchBytes, b->stream) != cudaSuccess) {
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return LBM_ERR_OOM;
  }
  *out = b;
  return LBM_OK;
}

lbm_status lbm_batch_add(lbm_batch *b, const int grid[3], const lbm_eos *eos, double G, const lbm_rates *rates, int op,
                         double sigma, int *id) {
  if (!b || !id) return LBM_ERR_ARG;
  if (!eos || eos->kind != b->eos) return bfail(b, LBM_ERR_ARG, "every box of a batch uses the batch's EOS kind");
  KParams P;
  if (op == LBM_OP_NONORTHOGONAL_D3Q15) return bfail(b, LBM_ERR_ARG, "batches hold D3Q19 boxes");
  if (!lbm::fill_params(grid, eos, G, rates, op, b->precision, sigma, &P)) return bfail(b, LBM_ERR_ARG, "bad box");
  const size_t bytes = box_bytes(b->precision, P.n);
  if (b->used + bytes > b->budget) return bfail(b, LBM_ERR_OOM, "HBM budget of the batch exceeded");
  HostBox h;
  BCK(cudaMallocAsync(&h.mem, bytes, b->stream), "box buffers");
  const size_t pop = (((size_t)19 * P.n * lbm::storage_bytes(b->precision)) + 255) / 256 * 256;
  const size_t ps = (((size_t)P.n * 4) + 255) / 256 * 256;
  char *m = (char *)h.mem;
  h.live = true;
  h.precision = b->precision;
  h.bytes = bytes;
  h.d.P = P;
  h.d.g[0] = m;
  h.d.g[1] = m + pop;
  h.d.psi[0] = (float *)(m + 2 * pop);
  h.d.psi[1] = (float *)(m + 2 * pop + ps);
  h.u_prev = (float *)(m + 2 * pop + 2 * ps);
  h.d.op = op;
  h.d.cur = b->phase;  // its state starts at level 0
  b->used += bytes;
  int slot = -1;
  for (int i = 0; i < (int)b->boxes.size(); ++i)
    if (!b->boxes[i].live) {
      slot = i;
      break;
    }
  if (slot < 0) {
    slot = (int)b->boxes.size();
    b->boxes.push_back(h);
  } else {
    b->boxes[slot] = h;
  }
  *id = slot;
  b->dirty = true;
  return LBM_OK;
}

lbm_status lbm_batch_remove(lbm_batch *b, int id) {
  HostBox *h = get_box(b, id);
  if (!h) return bfail(b, LBM_ERR_ARG, "no such box");
  cudaFreeAsync(h->mem, b->stream);
  b->used -= h->bytes;
  *h = HostBox();
  b->dirty = true;
  return LBM_OK;
}

lbm_status lbm_batch_init_droplet(lbm_batch *b, int id, const double centre[3], double R, double W, double rho_l,
                                  double rho_v) {
  HostBox *h = get_box(b, id);
  if (!h || !centre || !(W > 0) || !(rho_l > 0) || !(rho_v > 0) || !(R >= 0)) return bfail(b, LBM_ERR_ARG, "bad droplet");
  h->d.P.rho_ref = rho_v;
  lbm::refresh_float_params(h->d.P);
  lbm::DropletChunk ch{};
  ch.count = 1;
  ch.cx[0] = centre[0];
  ch.cy[0] = centre[1];
  ch.cz[0] = centre[2];
  ch.r[0] = R;
  double *rho = (double *)spare_g(b, h);
  BCK(lbm::launch_rho_droplets(h->d.P, rho, ch, W, rho_l, rho_v, true, launch_of(b)), "rho_droplets");
  return finish_box_init(b, h, rho);
}

lbm_status lbm_batch_init_flat(lbm_batch *b, int id, int axis, double lo, double hi, double W, double rho_l,
                               double rho_v) {
  HostBox *h = get_box(b, id);
  if (!h || axis < 0 || axis > 2 || !(lo < hi) || !(W > 0) || !(rho_l > 0) || !(rho_v > 0))
    return bfail(b, LBM_ERR_ARG, "bad slab");
  h->d.P.rho_ref = rho_v;
  lbm::refresh_float_params(h->d.P);
  double *rho = (double *)spare_g(b, h);
  BCK(lbm::launch_rho_slab(h->d.P, rho, axis, lo, hi, W, rho_l, rho_v, launch_of(b)), "rho_slab");
  return finish_box_init(b, h, rho);
}

lbm_status lbm_batch_set_tuning(lbm_batch *b, int tile, int id, int z_planes) {
  if (!b || tile < 0 || tile > kTileWorkList || z_planes < 0) return bfail(b, LBM_ERR_ARG, "bad tuning");
  b->tile = tile;
  if (id >= 0) {
    HostBox *h = get_box(b, id);
    if (!h) return bfail(b, LBM_ERR_ARG, "no such box");
    h->zc = z_planes;
  }
  b->dirty = true;
  return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch *b, int n) {
  if (!b || n < 1) return bfail(b, LBM_ERR_ARG, "n must be >= 1");
  if (b->dirty) {
    lbm_status s = rebuild(b);
    if (s != LBM_OK) return s;
  }
  if (!b->nitems) return LBM_OK;
  const char *name = b->wl ? (b->odd ? "lbm batch work-list + single pass (odd Nx)" : "lbm batch work-list step")
                    : b->pair ? (b->odd ? "lbm batch two-pass + single pass (odd Nx)" : "lbm batch two-pass step")
                              : "lbm batch single pass";
  for (int k = 0; k + 1 < n; k += 2) {
    const lbm::NvtxRange range(name);  // one graph: two steps
    BCK(cudaGraphLaunch(b->g2[b->phase], b->stream), "graph launch");
  }
  if (n & 1) {
    const lbm::NvtxRange range(name);
    BCK(cudaGraphLaunch(b->g1[b->phase], b->stream), "graph launch");
    b->phase ^= 1;  // every box's state is now at the other level
  }
  for (auto &h : b->boxes)
    if (h.live && h.initialised) h.steps += n;
  b->steps += n;
  return LBM_OK;
}

lbm_status lbm_batch_moments(lbm_batch *b, int id, double *rho, double *u, int on_device) {
  HostBox *h = get_box(b, id);
  if (!h || !h->initialised || (!rho && !u)) return bfail(b, LBM_ERR_ARG, "bad box or output");
  const lbm::Launch L = launch_of(b);
  const size_t n = h->d.P.n;
  if (on_device) {
    BCK(lbm::launch_moments(h->d.P, h->precision, cur_g(b, h), cur_psi(b, h), rho, u, L), "moments");
    return LBM_OK;
  }
  double *tmp = (double *)spare_g(b, h);  // 4N doubles fit in a population buffer
  BCK(lbm::launch_moments(h->d.P, h->precision, cur_g(b, h), cur_psi(b, h), tmp, tmp + n, L), "moments");
  if (rho) BCK(cudaMemcpyAsync(rho, tmp, sizeof(double) * n, cudaMemcpyDeviceToHost, b->stream), "D2H rho");
  if (u) BCK(cudaMemcpyAsync(u, tmp + n, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, b->stream), "D2H u");
  BCK(cudaStreamSynchronize(b->stream), "sync");
  return LBM_OK;
}

lbm_status lbm_batch_diag(lbm_batch *b, int id, double out[5]) {
  HostBox *h = get_box(b, id);
  if (!h || !h->initialised || !out) return bfail(b, LBM_ERR_ARG, "bad box or output");
  double *part = (double *)((char *)b->d_scratch + lbm::kScratchPartialOffset);
  double *res = (double *)((char *)b->d_scratch + lbm::kScratchResultOffset);
  BCK(lbm::launch_diag(h->d.P, h->precision, cur_g(b, h), cur_psi(b, h), part, res, launch_of(b)), "diag");
  BCK(cudaMemcpyAsync(out, res, 5 * sizeof(double), cudaMemcpyDeviceToHost, b->stream), "D2H diag");
  BCK(cudaStreamSynchronize(b->stream), "sync");
  return LBM_OK;
}

lbm_status lbm_batch_max_du(lbm_batch *b, int nid, const int *ids, double *out) {
  if (!b || nid < 0 || (nid && (!ids || !out))) return bfail(b, LBM_ERR_ARG, "bad arguments");
  if (nid > b->cap_red) {
    if (b->d_red) cudaFreeAsync(b->d_red, b->stream);
    BCK(cudaMallocAsync((void **)&b->d_red, sizeof(double) * nid, b->stream), "reduction buffer");
    b->cap_red = nid;
  }
  if (!nid) return LBM_OK;
  BCK(cudaMemsetAsync(b->d_red, 0, sizeof(double) * nid, b->stream), "clear");
  for (int k = 0; k < nid; ++k) {
    HostBox *h = get_box(b, ids[k]);
    if (!h || !h->initialised) return bfail(b, LBM_ERR_ARG, "bad box id");
    BCK(lbm::launch_max_du(h->d.P, h->precision, cur_g(b, h), cur_psi(b, h), h->u_prev, b->d_red + k, launch_of(b)),
        "max_du");
  }
  BCK(cudaMemcpyAsync(out, b->d_red, sizeof(double) * nid, cudaMemcpyDeviceToHost, b->stream), "D2H");
  BCK(cudaStreamSynchronize(b->stream), "sync");
  return LBM_OK;
}

lbm_status lbm_batch_check(lbm_batch *b) {
  if (!b) return LBM_ERR_ARG;
  unsigned w = 0;
  BCK(cudaMemcpyAsync(&w, b->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream), "read error word");
  BCK(cudaMemsetAsync(b->d_err, 0, sizeof(unsigned), b->stream), "clear error word");
  BCK(cudaStreamSynchronize(b->stream), "sync");
  if (lbm::dbg::take_all()) return bfail(b, LBM_ERR_BOUNDS, "a kernel index fell outside its buffer (debug build)");
  if (w & lbm::kErrTimeout) return bfail(b, LBM_ERR_TIMEOUT, "a bounded wait of the work-list step gave up");
  if (w & lbm::kErrNonFinite) return bfail(b, LBM_ERR_NONFINITE, "non-finite density");
  if (w & lbm::kErrEosDomain) return bfail(b, LBM_ERR_EOS_DOMAIN, "density left the domain of the EOS");
  return LBM_OK;
}

lbm_status lbm_batch_info(const lbm_batch *b, int *live_boxes, int *work_items, size_t *bytes_used) {
  if (!b) return LBM_ERR_ARG;
  int live = 0;
  for (auto &h : b->boxes) live += h.live ? 1 : 0;
  if (live_boxes) *live_boxes = live;
  if (work_items) *work_items = b->nitems;
  if (bytes_used) *bytes_used = b->used;
  return LBM_OK;
}

long long lbm_batch_graph_builds(const lbm_batch *b) { return b ? b->builds : -1; }

long long lbm_batch_box_steps(const lbm_batch *b, int id) {
  if (!b || id < 0 || id >= (int)b->boxes.size() || !b->boxes[id].live) return -1;
  return b->boxes[id].steps;
}

const char *lbm_batch_last_error(const lbm_batch *b) { return b ? b->err.c_str() : ""; }

void lbm_batch_destroy(lbm_batch *b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  destroy_graphs(b);
  for (auto &h : b->boxes)
    if (h.live) cudaFreeAsync(h.mem, b->stream);
  if (b->d_boxes) cudaFreeAsync(b->d_boxes, b->stream);
  if (b->d_items) cudaFreeAsync(b->d_items, b->stream);
  if (b->d_red) cudaFreeAsync(b->d_red, b->stream);
  if (b->d_done) cudaFreeAsync(b->d_done, b->stream);
  if (b->d_fmap) cudaFreeAsync(b->d_fmap, b->stream);
  if (b->d_err) cudaFreeAsync(b->d_err, b->stream);
  if (b->d_scratch) cudaFreeAsync(b->d_scratch, b->stream);
  cudaStreamSynchronize(b->stream);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
}

}  // extern "C"
