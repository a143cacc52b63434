// Internal interface between the C ABI (lbm_api.cu) and the kernels
// (lbm_kernels.cu).  Not installed; not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <vector>

namespace lbm {

enum Precision { kF64 = 0, kF32 = 1, kF16 = 2 };
enum Operator { kOrth = 0, kNonOrth = 1, kNonOrthQ15 = 2 };
enum EosKind { kEosCS = 0, kEosExp = 1, kEosNone = 2 };

// Error bits the kernels set in the device error word.
enum : unsigned { kErrEosDomain = 1u, kErrNonFinite = 2u, kErrTimeout = 4u };

// Everything a kernel needs about the box and the physics, passed by value.
struct KParams {
  int nx, ny, nz;
  int n;             // nx * ny * nz (< 2^31)
  int q;             // lattice: 19 (D3Q19, both operators) or 15 (D3Q15 non-orthogonal)
  double G;          // interaction strength, Eq. 15
  double rho_ref;    // reference density of the deviation storage
  // relaxation rates (see lbm_rates in lbm.h)
  double s_e, s_nu, s_q, s_pi, s_eps, s_m;
  // Eq. 16 coefficient: the extra S_4 is sigma_coef * |sum_a w_a psi(x+e_a) e_a|^2
  // (= 6 sigma |F|^2 / (psi^2 (1/s_e - 1/2)) with F = -G psi sum(...)).
  double sigma_coef;
  // equation of state
  int eos;
  double a, b, RT;   // Carnahan-Starling (Eq. 58), RT = R * T
  double psi0, rho0; // exponential pseudopotential
  double b4;         // b / 4
  double two_over_G; // 2 / G
  // (2/G) (RT num - (a rho + 1/3) den) = q0 + q1 rho + q2 rho^2 + q3 rho^3 + q4 rho^4,
  // num = 1 + eta + eta^2 - eta^3, den = (1 - eta)^3, eta = b rho / 4 (Eq. 58)
  double q0, q1, q2, q3, q4;
  float f_rho_max;   // 4 / b: the packing limit eta < 1
  // FP32 copies for the reduced-precision kernels (no conversions on device)
  float fG, frho_ref, fs_e, fs_nu, fs_q, fs_pi, fs_eps, fs_m, fsigma_coef, fb4;
  // density-dependent shear viscosity: nu(rho) = nu_v + (rho - rho_v) nu_slope,
  // clamped to [nu_lo, nu_hi]; s_nu(rho) = 1 / (3 nu + 1/2).  Off unless varnu.
  int varnu;
  double nu_v, rho_v_nu, nu_slope, nu_lo, nu_hi;
  float fnu_v, frho_v_nu, fnu_slope, fnu_lo, fnu_hi;
  // the radicand coefficients and rho_ref as unevaluated sums of two floats
  // (hi + lo), for the compensated-FP32 evaluation of the EOS
  float qh[5], ql[5], rr_h, rr_l;
  // the same radicand as a quintic in d = rho - rho_ref: sum_k c[k] d^k
  double c[6];
  // bounded device-side waits (single-pass kernels): polls before a wait gives
  // up and sets kErrTimeout; wait_bias is added to every cross-block wait
  // target (0; 1 makes the targets unreachable, a host-side fault injection)
  int spin_limit;
  int wait_bias;
};

constexpr int kDefaultSpinLimit = 1 << 22;

// An NVTX range around a scope (a kernel launch, a graph launch): visible in
// profilers that trace NVTX; a cheap no-op otherwise.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// Layout of the scratch buffer.
constexpr int kReduceBlocks = 1024;
constexpr size_t kScratchErrOffset = 0;      // unsigned error word
constexpr size_t kScratchPartialOffset = 256;  // kReduceBlocks x 5 doubles
constexpr size_t kScratchResultOffset = kScratchPartialOffset + sizeof(double) * 5 * kReduceBlocks;
constexpr size_t kScratchBytes = kScratchResultOffset + 256;

// Droplets handed to the density-field kernel in chunks.
constexpr int kDropletChunk = 64;
struct DropletChunk {
  int count;
  double cx[kDropletChunk], cy[kDropletChunk], cz[kDropletChunk], r[kDropletChunk];
};

struct Launch {
  cudaStream_t stream;
  int bx, by;  // thread-block shape (x, y) of the per-node kernels
};

// Fill the FP32 copies of KParams from its doubles (call after any change).
inline void refresh_float_params(KParams &P) {
  P.fG = (float)P.G;
  P.frho_ref = (float)P.rho_ref;
  P.fs_e = (float)P.s_e;
  P.fs_nu = (float)P.s_nu;
  P.fs_q = (float)P.s_q;
  P.fs_pi = (float)P.s_pi;
  P.fs_eps = (float)P.s_eps;
  P.fs_m = (float)P.s_m;
  P.fsigma_coef = (float)P.sigma_coef;
  P.fb4 = (float)P.b4;
  const double q[5] = {P.q0, P.q1, P.q2, P.q3, P.q4};
  for (int k = 0; k < 5; ++k) {
    P.qh[k] = (float)q[k];
    P.ql[k] = (float)(q[k] - (double)P.qh[k]);
  }
  P.fnu_v = (float)P.nu_v;
  P.frho_v_nu = (float)P.rho_v_nu;
  P.fnu_slope = (float)P.nu_slope;
  P.fnu_lo = (float)P.nu_lo;
  P.fnu_hi = (float)P.nu_hi;
  P.rr_h = (float)P.rho_ref;
  P.rr_l = (float)(P.rho_ref - (double)P.rr_h);
  // X(rho) = sum_{m=1..5} q[m-1] rho^m with rho = rho_ref + d:
  // c[k] = sum_{m >= max(k, 1)} q[m-1] binom(m, k) rho_ref^(m-k)
  static const double binom[6][6] = {{1, 0, 0, 0, 0, 0},  {1, 1, 0, 0, 0, 0},   {1, 2, 1, 0, 0, 0},
                                     {1, 3, 3, 1, 0, 0},  {1, 4, 6, 4, 1, 0},   {1, 5, 10, 10, 5, 1}};
  for (int k = 0; k <= 5; ++k) {
    double acc = 0.0;
    for (int m = k > 1 ? k : 1; m <= 5; ++m) {
      double rp = 1.0;
      for (int j = 0; j < m - k; ++j) rp *= P.rho_ref;
      acc += q[m - 1] * binom[m][k] * rp;
    }
    P.c[k] = acc;
  }
}

// x-y tile shapes of the single-pass kernel.
enum Tile { kTile32x4 = 0, kTile32x8 = 1, kTile64x4 = 2 };

// Single-pass step (FP32 and FP16-storage forms): reads populations g_in and
// psi(t) from psi_in, writes populations g_out and psi(t+1) to psi_out.  zc is
// the number of z planes each CTA marches through.
cudaError_t launch_onepass(const KParams &P, int precision, int op, bool sigma, int tile, int zc, const void *g_in,
                           void *g_out, const void *psi_in, void *psi_out, unsigned *err, cudaStream_t s);

// One box of a batch as the batched kernel sees it (copied to shared memory
// per work item).  g[k] / psi[k]: the two time levels; cur: which level holds
// the state at the batch's parity 0.
struct alignas(16) BatchBox {  // 16-byte aligned: copied to shared memory in 16-byte pieces
  KParams P;
  void *g[2];
  float *psi[2];
  int op;
  int cur;
  int qbase;  // first completion counter of this box in the batch work list, or (two-pass step) its first
              // block of the flat fused grid
  int tw;     // its tile width there (batch_tile_width)
  // the rest of its work-list tile geometry (batch_queue_geometry): tiles along x and y and per plane, tile
  // height, log2 of the node pairs across a tile, and ntx_m = ceil(2^32 / ntx), so that t / ntx is
  // (t * ntx_m) >> 32 for every tile index t < 2^16
  int ntx, nty, T, th, hshift;
  unsigned long long ntx_m;
};

// Persistent single-pass launch over the work items (box, tx | ty << 16, z0, z1)
// of many boxes; grid = number of thread blocks.  FP32 arithmetic forms only.
// The batch's two-pass step on the pair kernels (every box with an even Nx):
// the fused pass, then the psi pass of the new level, for one parity.  The
// fused pass is a flat grid per operator, one block per plane of a tile of the
// chosen shape: block_box holds the box of every block, the non-orthogonal
// boxes' fused_blocks[0] blocks first, then the orthogonal boxes'
// fused_blocks[1]; a box's blocks are consecutive from its descriptor's qbase,
// plane by plane, tiles x-fastest.  The psi pass is a persistent grid of
// sms x per_sm[1] blocks over the items (at most one per item), per_sm as
// batch_pair_occupancy gives it (resident blocks per SM; [0] is unused).
cudaError_t batch_pair_occupancy(int precision, int eos, int tile, int per_sm[2]);
cudaError_t launch_batch_pair(int precision, int eos, int tile, const BatchBox *boxes, const int4 *items, int nitems,
                              const int *block_box, const int fused_blocks[2], int parity, int sms,
                              const int per_sm[2], unsigned *err, cudaStream_t s);
cudaError_t launch_batch_onepass(int precision, int eos, int tile, const BatchBox *boxes, const int4 *items,
                                 int nitems, int parity, int grid, unsigned *err, cudaStream_t s);
// Block shape of a tile choice: returns threads per block, sets bx, by.
int onepass_tile_shape(int tile, int *bx, int *by);

// Single-pass step whose data movement runs on bulk asynchronous copies
// (FP32 storage, 32x8 tiles, nx % 4 == 0 and nx >= 40).
bool onepass_tma_supported(const KParams &P, int precision);
cudaError_t launch_onepass_tma(const KParams &P, int precision, int op, bool sigma, int zc, const void *g_in,
                               void *g_out, const void *psi_in, void *psi_out, unsigned *err, cudaStream_t s);

// Two-pass kernels of the FP32-arithmetic forms with two x-adjacent nodes per
// thread and packed FP32 arithmetic (Nx even).
bool pair_supported(const KParams &P, int precision);
cudaError_t launch_psi_pair(const KParams &P, int precision, const void *g, void *psi, unsigned *err,
                            const Launch &L, bool df);
cudaError_t launch_fused_pair(const KParams &P, int precision, int op, bool sigma, const void *g_in, void *g_out,
                              const void *psi, const Launch &L);

// Single-pass step with psi evaluated on chip by producer warps and the
// collision run by consumer warps (FP32 arithmetic, Nx even); no psi array.
bool onchip_supported(const KParams &P, int precision);
cudaError_t launch_onchip(const KParams &P, int precision, int op, bool sigma, bool df, const void *g_in, void *g_out,
                          unsigned *err, cudaStream_t s);

// Single-pass step in which psi of the next step trails the fused pass by one
// plane in one cooperative launch (FP32 arithmetic, Nx even).  flags: an int
// per (tile, plane), lagged_flag_count(P) of them, zero before the first
// launch; stamp: a number larger than in every earlier launch on these flags.
bool lagged_supported(const KParams &P, int precision);
size_t lagged_flag_count(const KParams &P);
cudaError_t launch_lagged(const KParams &P, int precision, int op, bool sigma, bool df, const void *g_in, void *g_out,
                          const void *psi_in, void *psi_out, int *flags, int stamp, unsigned *err, cudaStream_t s);

// Single-pass step on an ordered work list (FP32 arithmetic, D3Q19, Nx even):
// items of a fused tile job and a lagging psi tile job, one cooperative launch
// of `grid` blocks (queue_grid) working through the list queue_items builds
// (and checks: false if it cannot).  The device side: the item table, a
// completion counter per fused job and the blocks' item-claim counter
// (queue_counters ints, zero before the first launch).
struct QueueState {
  const int4 *items;
  int nitems;
  int grid;
  int *done;
};
bool queue_supported(const KParams &P, int precision);
cudaError_t queue_grid(int precision, int *grid);
size_t queue_counters(const KParams &P);
bool queue_items(const KParams &P, int grid, std::vector<int4> &out);
// stamp: 1 + the number of earlier launches on these counters.
cudaError_t launch_queue(const KParams &P, int precision, int op, bool sigma, bool df, const void *g_in, void *g_out,
                         const void *psi_in, void *psi_out, const QueueState &q, int stamp, unsigned *err,
                         cudaStream_t s);

// The work-list step over a batch (every box D3Q19 with an even Nx): one
// cooperative launch per step; items hold a fused tile job and a psi tile job
// of any boxes (x / z: box index or -1, y / w: z | tile << 16).  The list is
// built for the boxes in the given order; base[k] receives box k's first
// completion counter, *ncounters their total.  Counters must be zero when a
// launch starts (the step graph clears them).
bool batch_queue_items(const std::vector<const KParams *> &boxes, int grid, std::vector<int4> &out,
                       std::vector<int> &base, long long *ncounters);
int batch_tile_width(int nx);               // 64, 32 or 16: tiles of tw x (256 / tw) nodes
void batch_queue_geometry(BatchBox &d);     // sets d.tw and the geometry fields from d.P
int batch_queue_tiles(const KParams &P);   // tile jobs per plane of a box in a batch work list
cudaError_t batch_queue_grid(int precision, int eos, int *grid);
cudaError_t launch_batch_queue(int precision, int eos, const BatchBox *boxes, const int4 *items, int nitems,
                               int parity, int grid, int *done, int ndone, unsigned *err, cudaStream_t s);

// Debug build (-DLBM_BOUNDS_CHECK): OR of the bounds-error words of every
// translation unit, each cleared (synchronous); 0 in the normal build.
namespace dbg {
unsigned take_all();
}

size_t storage_bytes(int precision);  // bytes per stored population
size_t psi_elem_bytes(int precision);

// One time step is launch_psi followed by launch_fused (buffers swapped by the caller).
// df: evaluate the EOS radicand in compensated FP32 pairs (FP32 / FP16 forms)
cudaError_t launch_psi(const KParams &P, int precision, const void *g, void *psi,
                       unsigned *err, const Launch &L, bool df = false);
cudaError_t launch_fused(const KParams &P, int precision, int op, bool sigma,
                         const void *g_in, void *g_out, const void *psi, const Launch &L);

cudaError_t launch_moments(const KParams &P, int precision, const void *g, const void *psi,
                           double *rho, double *u, const Launch &L);
cudaError_t launch_diag(const KParams &P, int precision, const void *g, const void *psi,
                        double *partials, double *result, const Launch &L);

// max |u - u_prev| over the box into *out (atomic max; *out must start at 0), u_prev := u.
cudaError_t launch_max_du(const KParams &P, int precision, const void *g, const void *psi, float *u_prev,
                          double *out, const Launch &L);
cudaError_t launch_rho_droplets(const KParams &P, double *rho, const DropletChunk &chunk,
                                double W, double rho_l, double rho_v, bool first, const Launch &L);
cudaError_t launch_rho_slab(const KParams &P, double *rho, int axis, double lo, double hi,
                            double W, double rho_l, double rho_v, const Launch &L);
cudaError_t launch_state_from_rho(const KParams &P, int precision, const double *rho, void *g,
                                  const Launch &L);
cudaError_t launch_get_populations(const KParams &P, int precision, const void *g, double *out,
                                   int a_lo, int a_hi, const Launch &L);
cudaError_t launch_set_populations(const KParams &P, int precision, const double *f, void *g,
                                   int a_lo, int a_hi, const Launch &L);

}  // namespace lbm
