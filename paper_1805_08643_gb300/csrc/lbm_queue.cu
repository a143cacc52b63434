// Single-pass time step on an ordered work list (FP32-arithmetic forms, D3Q19,
// Nx even): one persistent launch per step runs both passes of the two-pass
// step as interleaved work.
//
// Work item k is a pair of tile jobs (64 x 4 nodes of one plane, one node
// pair per thread):
//   fused job (z, tile): the fused pass (Eqs. 4-6 and 15, pull streaming of
//     Eq. 5): reads f(t) and psi(t), writes f*(t); then counts itself done;
//   psi job (z', tile'): the psi pass of the next step: rho(t+1) from the
//     pulled f*(t) (Eq. 6), the EOS, psi(t+1).  It needs the fused jobs of
//     planes z'-1..z'+1 on the tile and its eight neighbours (periodic) and
//     pulls their output through L2, where it still is.
// The host builds the list (and checks it): fused jobs plane by plane; each
// psi job in the first free item at least half a wave of the grid (grid / 2
// items) after the last fused job it reads.  Half a wave: by the time a block
// reaches the psi job those fused jobs are normally finished, so the wait is
// one poll, while writer and reader stay close enough for the populations to
// be still in L2 (measured on GB300: a whole wave waits less but re-reads about
// twice as much from DRAM, and is slower; a quarter waits more).
//
// Block b starts with item b; from then on it claims the next unclaimed item
// (one atomic fetch per item, issued when an item starts and read when it
// ends), so blocks take items in list order whatever their speed.  (With the
// static order b, b + grid, ..., blocks drifted up to five items apart within
// a wave, and the psi jobs of the fast ones waited on the slow ones: 0.556
// against 0.528 ms per 256^3 step on GB300.)  Claims are in increasing order
// and the launch is cooperative (every block resident): a block holding an
// unfinished fused job is busy with an earlier item, so the psi job of the
// lowest unfinished item waits only on fused jobs that are finished or
// running, and progress needs no timing assumption.  Waits are bounded all
// the same (KParams::spin_limit; a wait that gives up sets kErrTimeout and
// the launch still ends).
//
// What this buys over two launches: the psi jobs' FP64 EOS runs on the same
// SMs while the fused jobs stream HBM, and the populations they pull come from
// L2 (writer and reader are about two planes plus half a wave of tiles apart): DRAM traffic per node is f(t) read and f*(t) written once plus psi
// read and written once (2 x 19 x s + 8 bytes) against 3 x 19 x s + 8.  The
// arithmetic and its order are those of the two-pass kernels, so the results
// are equal bit for bit.
//
// Counters: done[z * T + tile] counts the launches in which fused job
// (z, tile) has finished (one release increment after a block barrier), so a
// psi job of launch `stamp` waits for done >= stamp and nothing is ever reset.
// done[nz * T + 16] counts the item claims: exactly nitems per launch (one
// for every item a block runs; the one made during a block's last item names
// no item), so launch `stamp` claims numbers (stamp - 1) * nitems onwards,
// modulo 2^32.
#include <cuda_fp16.h>

#include <algorithm>
#include <vector>

#include "lbm_device.cuh"
#include "lbm_internal.h"
#include "lbm_pair.cuh"
#include "lbm_pair15.cuh"

namespace lbm {
namespace {

constexpr int TXP = 32;          // pair columns of a tile: 64 nodes
constexpr int kRows = 4;         // rows of a tile (one warp each)
constexpr int NTH = TXP * kRows;
constexpr int kMinBlocks = 6;    // resident blocks per SM the register budget is set for
// The psi jobs convert to and from FP64 with the conversion instructions, not
// the integer path of the psi pass kernel (the same results): this kernel is
// not bound by the FP64 unit, and the integer work cost 1 % (FP32 storage) and
// 3 % (FP16) of a 256^3 step on GB300.
constexpr bool kIntCvt = false;

struct TileGeo {
  int ntx, nty, T;  // tiles along x, along y, per plane
};

__host__ __device__ inline TileGeo tile_geo(const KParams &P) {
  TileGeo g;
  g.ntx = (P.nx + 2 * TXP - 1) / (2 * TXP);
  g.nty = (P.ny + kRows - 1) / kRows;
  g.T = g.ntx * g.nty;
  return g;
}

// The item claim number c of this launch names: gridDim.x + c.  Every launch
// makes exactly nitems claims, so c < nitems; a claim outside that range
// (claim counter and launch count out of step) ends the block's loop and is
// reported as a timeout: the list could not be followed.
__device__ __forceinline__ int next_item(unsigned c, int nitems, unsigned &e) {
  if (c >= (unsigned)nitems) {
    e |= kErrTimeout;
    return nitems;
  }
  return (int)gridDim.x + (int)c;
}

// item: x = fused plane (or -1), y = its tile, z = psi plane (or -1), w = its tile.
// Q: 19 (both operators) or 15 (the D3Q15 non-orthogonal variant).
template <typename S, int OP, bool SIGMA, int EOS, bool DF, int Q>
__global__ void __launch_bounds__(NTH, kMinBlocks)
    queue_kernel(const S *__restrict__ g_in, S *__restrict__ g_out, const float *__restrict__ psi_in,
                 float *__restrict__ psi_out, const KParams P, const int4 *__restrict__ items, int nitems,
                 int *__restrict__ done, int stamp, unsigned *__restrict__ err) {
  const TileGeo G = tile_geo(P);
  const int lane = threadIdx.x, row = threadIdx.y;
  unsigned e = 0;
  // the claimed next item, by item parity: thread 0 writes slot i & 1 before item i's barrier and the block
  // reads it after that barrier; the slot is written again two items later, after every thread has passed
  // item i + 1's barrier
  __shared__ int s_next[2];
  unsigned *claims = (unsigned *)(done + P.nz * G.T + 16);
  const unsigned base = (unsigned)(stamp - 1) * (unsigned)nitems;
  int k = blockIdx.x;
  int par = 0;
#pragma unroll 1
  while (k < nitems) {
    unsigned claim = 0;
    if (lane == 0 && row == 0) claim = atomicAdd(claims, 1u);  // the next item: gridDim.x + claim - base
    const int4 it = __ldg(items + k);
    if (it.x >= 0) {
      int z = it.x, t = it.y;
      asm volatile("" : "+r"(z), "+r"(t));  // keep the row offsets out of the registers across items
      const int x = (t % G.ntx) * 2 * TXP + 2 * lane, y = (t / G.ntx) * kRows + row;
      if (x < P.nx && y < P.ny) {
        if constexpr (Q == 15)
          fused_pair15_at<S, SIGMA>(g_in, g_out, psi_in, P, x, y, z);
        else
          fused_pair_at<S, OP, SIGMA, false>(g_in, g_out, psi_in, P, x, y, z, Rates<V2>(P));
      }
      if (lane == 0 && row == 0) s_next[par] = next_item(claim - base, nitems, e);
      __syncthreads();
      if (lane == 0 && row == 0) counter_release_add(done + LBM_IDX(z * G.T + t, P.nz * G.T), 1);
    } else {
      if (lane == 0 && row == 0) s_next[par] = next_item(claim - base, nitems, e);
      __syncthreads();
    }
    const int kn = s_next[par];
    par ^= 1;
    if (it.z >= 0) {
      int z = it.z, t = it.w;
      asm volatile("" : "+r"(z), "+r"(t));
      const int tx = t % G.ntx, ty = t / G.ntx;
      bool ok = true;
      if (lane < 27) {  // fused jobs of planes z-1..z+1 on the 3 x 3 tiles around (tx, ty)
        int zz = z + lane / 9 - 1, xx = tx + lane % 3 - 1, yy = ty + (lane / 3) % 3 - 1;
        zz = zz < 0 ? zz + P.nz : (zz >= P.nz ? zz - P.nz : zz);
        xx = xx < 0 ? xx + G.ntx : (xx >= G.ntx ? xx - G.ntx : xx);
        yy = yy < 0 ? yy + G.nty : (yy >= G.nty ? yy - G.nty : yy);
        const int *c = done + LBM_IDX(zz * G.T + yy * G.ntx + xx, P.nz * G.T);
        const int target = stamp + P.wait_bias;
        for (int n = 0; counter_acquire(c) < target; ++n) {
          if (n >= P.spin_limit) {
            ok = false;
            break;
          }
          __nanosleep(32);
        }
      }
      if (!__all_sync(0xffffffffu, ok)) e |= kErrTimeout;
      const int x = tx * 2 * TXP + 2 * lane, y = ty * kRows + row;
      if (x < P.nx && y < P.ny) {
        if constexpr (Q == 15)
          psi_pair15_at_l2<S, EOS, DF, kIntCvt>(g_out, psi_out, P, x, y, z, e);
        else
          psi_pair_at_l2<S, EOS, DF, kIntCvt>(g_out, psi_out, P, x, y, z, e);
      }
    }
    k = kn;
  }
  if (e) atomicOr(err, e);
}

template <typename S, int OP, bool SIGMA, int EOS, bool DF, int Q>
cudaError_t launch_kernel(const KParams &P, const void *g_in, void *g_out, const void *psi_in, void *psi_out,
                          const QueueState &q, int stamp, unsigned *err, cudaStream_t s) {
  auto kern = queue_kernel<S, OP, SIGMA, EOS, DF, Q>;
  const S *gi = (const S *)g_in;
  S *go = (S *)g_out;
  const float *pi = (const float *)psi_in;
  float *po = (float *)psi_out;
  KParams Pc = P;
  const int4 *items = q.items;
  int nitems = q.nitems, *done = q.done;
  void *args[] = {(void *)&gi,    (void *)&go,     (void *)&pi,   (void *)&po,    (void *)&Pc,
                  (void *)&items, (void *)&nitems, (void *)&done, (void *)&stamp, (void *)&err};
  return cudaLaunchCooperativeKernel((const void *)kern, dim3(q.grid), dim3(TXP, kRows), args, 0, s);
}

template <typename S, int OP, bool SIGMA, int Q = 19>
cudaError_t by_eos(const KParams &P, bool df, const void *g_in, void *g_out, const void *psi_in, void *psi_out,
                   const QueueState &q, int stamp, unsigned *err, cudaStream_t s) {
  switch (P.eos) {
    case kEosCS:
      return df ? launch_kernel<S, OP, SIGMA, kEosCS, true, Q>(P, g_in, g_out, psi_in, psi_out, q, stamp, err, s)
                : launch_kernel<S, OP, SIGMA, kEosCS, false, Q>(P, g_in, g_out, psi_in, psi_out, q, stamp, err, s);
    case kEosExp:
      return df ? launch_kernel<S, OP, SIGMA, kEosExp, true, Q>(P, g_in, g_out, psi_in, psi_out, q, stamp, err, s)
                : launch_kernel<S, OP, SIGMA, kEosExp, false, Q>(P, g_in, g_out, psi_in, psi_out, q, stamp, err, s);
    default:
      return launch_kernel<S, OP, SIGMA, kEosNone, false, Q>(P, g_in, g_out, psi_in, psi_out, q, stamp, err, s);
  }
}

template <typename S>
cudaError_t by_op(const KParams &P, int op, bool sigma, bool df, const void *g_in, void *g_out, const void *psi_in,
                  void *psi_out, const QueueState &q, int stamp, unsigned *err, cudaStream_t s) {
  if (P.q == 15)
    return sigma ? by_eos<S, kNonOrth, true, 15>(P, df, g_in, g_out, psi_in, psi_out, q, stamp, err, s)
                 : by_eos<S, kNonOrth, false, 15>(P, df, g_in, g_out, psi_in, psi_out, q, stamp, err, s);
  if (op == kNonOrth)
    return sigma ? by_eos<S, kNonOrth, true>(P, df, g_in, g_out, psi_in, psi_out, q, stamp, err, s)
                 : by_eos<S, kNonOrth, false>(P, df, g_in, g_out, psi_in, psi_out, q, stamp, err, s);
  return sigma ? by_eos<S, kOrth, true>(P, df, g_in, g_out, psi_in, psi_out, q, stamp, err, s)
               : by_eos<S, kOrth, false>(P, df, g_in, g_out, psi_in, psi_out, q, stamp, err, s);
}

// Resident blocks per SM of the kernels a context launches: the smallest over
// the instantiations of the storage type, so that a cooperative launch of
// that many blocks per SM fits whichever one runs.
template <typename S>
cudaError_t occupancy_of(int *per_sm) {
  using K = void (*)(const S *, S *, const float *, float *, const KParams, const int4 *, int, int *, int, unsigned *);
  const K ks[] = {queue_kernel<S, kNonOrth, true, kEosCS, false, 19>, queue_kernel<S, kOrth, true, kEosCS, false, 19>,
                  queue_kernel<S, kNonOrth, false, kEosCS, true, 19>, queue_kernel<S, kOrth, false, kEosExp, false, 19>,
                  queue_kernel<S, kNonOrth, true, kEosCS, false, 15>, queue_kernel<S, kNonOrth, false, kEosExp, true, 15>};
  int m = 1 << 30;
  for (K k : ks) {
    int v = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k, NTH, 0);
    if (e != cudaSuccess) return e;
    m = std::min(m, v);
  }
  *per_sm = m;
  return cudaSuccess;
}

// ------------------------------------------------------------------ batches
// The same work list over many boxes.  Every job carries its box, whose
// descriptor (parameters, buffers, operator, level, tile width) the block
// copies to shared memory one item ahead (asynchronous copies, double
// buffered), so it is there when the item starts; a fused job of box B
// reads level in = B.cur ^ parity and writes in ^ 1, the psi job evaluates psi
// of level in ^ 1.  Both operators and the Eq. 16 term (zero coefficient when
// off) are compiled in.  Tiles are tw x (256 / tw) nodes, tw = 64, 32 or 16 per
// box (batch_tile_width): 128 threads, one node pair each, and on the small
// boxes of a batch (edges 32, 48, 96, ...) no idle half tiles.
struct BatchGeo {
  int tw, th, ntx, nty, T;  // tile width and height, tiles along x and y, per plane
};

__host__ __device__ inline BatchGeo batch_geo(const KParams &P, int tw) {
  BatchGeo g;
  g.tw = tw;
  g.th = 2 * NTH / tw;
  g.ntx = (P.nx + tw - 1) / tw;
  g.nty = (P.ny + g.th - 1) / g.th;
  g.T = g.ntx * g.nty;
  return g;
}

// Tile row of tile t of a box: t / ntx by a multiply with the descriptor's
// ceil(2^32 / ntx) instead of a division (exact for t * ntx < 2^32).
__device__ __forceinline__ int tile_row(int t, const BatchBox &B) {
  return (int)(((unsigned long long)(unsigned)t * B.ntx_m) >> 32);
}

// Copy box descriptors to shared memory with asynchronous 16-byte copies (one
// commit group per call), so that the next item's descriptors arrive while the
// current item runs.
__device__ __forceinline__ void prefetch_boxes(BatchBox *dst, const BatchBox *__restrict__ boxes, int4 it, int tid,
                                               int nthreads = NTH) {
  constexpr int chunks = (int)(sizeof(BatchBox) / 16);
  static_assert(sizeof(BatchBox) % 16 == 0, "descriptor copies move 16-byte pieces");
  for (int side = 0; side < 2; ++side) {
    const int box = side ? it.z : it.x;
    if (box < 0) continue;
    const char *src = (const char *)(boxes + box);
    char *d = (char *)(dst + side);
    for (int c = tid; c < chunks; c += nthreads) {
      const unsigned sa = (unsigned)__cvta_generic_to_shared(d + 16 * c);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(src + 16 * c) : "memory");
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

template <typename S, int EOS>
__global__ void __launch_bounds__(NTH, kMinBlocks)
    batch_queue_kernel(const BatchBox *__restrict__ boxes, const int4 *__restrict__ items, int nitems, int parity,
                       int *__restrict__ done, int ndone, unsigned *__restrict__ err) {
  __shared__ BatchBox bb[2][2];  // [item parity][fused job's box, psi job's box]
  const int tid = threadIdx.y * TXP + threadIdx.x;
  unsigned e = 0;
  // block b starts with item b, then claims the next unclaimed item (one atomic fetch per item, issued
  // when an item starts); warp 0 reads the claimed item and copies its descriptors during the psi job
  __shared__ int s_next;
  __shared__ int4 s_it;
  unsigned *claims = (unsigned *)(done + ndone + 16);  // cleared with the counters before every launch
  int k = blockIdx.x;
  int4 it = k < nitems ? __ldg(items + k) : make_int4(-1, -1, -1, -1);
  prefetch_boxes(bb[0], boxes, it, tid);
#pragma unroll 1
  for (int i = 0; k < nitems; ++i) {
    unsigned claim = 0;
    if (tid == 0) claim = atomicAdd(claims, 1u);  // the next item: gridDim.x + claim
    asm volatile("cp.async.wait_group 0;" ::: "memory");  // this item's descriptors have arrived
    __syncthreads();
    if (it.x >= 0) {
      const BatchBox &B = bb[i & 1][0];
      const KParams &P = B.P;
      int z = (int)((unsigned)it.y & 0xffffu), t = (int)((unsigned)it.y >> 16);
      asm volatile("" : "+r"(z), "+r"(t));
      const int in = B.cur ^ parity;
      const int ty = tile_row(t, B), tx = t - ty * B.ntx;
      const int x = tx * B.tw + 2 * (tid & ((1 << B.hshift) - 1)), y = ty * B.th + (tid >> B.hshift);
      if (x < P.nx && y < P.ny) {
        const S *gi = (const S *)B.g[in];
        S *go = (S *)B.g[in ^ 1];
        if (B.op == kNonOrth)
          fused_pair_at<S, kNonOrth, true, false>(gi, go, B.psi[in], P, x, y, z, Rates<V2>(P));
        else
          fused_pair_at<S, kOrth, true, false>(gi, go, B.psi[in], P, x, y, z, Rates<V2>(P));
      }
      __syncthreads();
      if (tid == 0) counter_release_add(done + LBM_IDX(B.qbase + z * B.T + t, ndone), 1);
    }
    if (threadIdx.y == 0) {  // the next item and its descriptors (buffer (i + 1) & 1 was item i - 1's)
      const int kn = (int)min((unsigned)gridDim.x + __shfl_sync(0xffffffffu, claim, 0), (unsigned)nitems);
      const int4 nx = kn < nitems ? __ldg(items + kn) : make_int4(-1, -1, -1, -1);
      prefetch_boxes(bb[(i + 1) & 1], boxes, nx, threadIdx.x, TXP);
      if (threadIdx.x == 0) {
        s_next = kn;
        s_it = nx;
      }
    }
    if (it.z >= 0) {
      const BatchBox &B = bb[i & 1][1];
      const KParams &P = B.P;
      int z = (int)((unsigned)it.w & 0xffffu), t = (int)((unsigned)it.w >> 16);
      asm volatile("" : "+r"(z), "+r"(t));
      const int ty = tile_row(t, B), tx = t - ty * B.ntx, lane = threadIdx.x;
      bool ok = true;
      if (lane < 27) {  // fused jobs of planes z-1..z+1 on the 3 x 3 tiles around (tx, ty)
        int zz = z + lane / 9 - 1, xx = tx + lane % 3 - 1, yy = ty + (lane / 3) % 3 - 1;
        zz = zz < 0 ? zz + P.nz : (zz >= P.nz ? zz - P.nz : zz);
        xx = xx < 0 ? xx + B.ntx : (xx >= B.ntx ? xx - B.ntx : xx);
        yy = yy < 0 ? yy + B.nty : (yy >= B.nty ? yy - B.nty : yy);
        const int *c = done + LBM_IDX(B.qbase + zz * B.T + yy * B.ntx + xx, ndone);
        const int target = 1 + P.wait_bias;  // counters are cleared before every launch
        for (int n = 0; counter_acquire(c) < target; ++n) {
          if (n >= P.spin_limit) {
            ok = false;
            break;
          }
          __nanosleep(32);
        }
      }
      if (!__all_sync(0xffffffffu, ok)) e |= kErrTimeout;
      const int in = B.cur ^ parity;
      const int x = tx * B.tw + 2 * (tid & ((1 << B.hshift) - 1)), y = ty * B.th + (tid >> B.hshift);
      if (x < P.nx && y < P.ny) psi_pair_at_l2<S, EOS, false, kIntCvt>((const S *)B.g[in ^ 1], B.psi[in ^ 1], P, x, y, z, e);
    }
    __syncthreads();  // s_next and s_it are written; rewritten only after the next item's first barrier
    k = s_next;
    it = s_it;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");  // no copy outlives the block
  if (e) atomicOr(err, e);
}

template <typename S, int EOS>
cudaError_t batch_launch(const BatchBox *boxes, const int4 *items, int nitems, int parity, int grid, int *done,
                         int ndone, unsigned *err, cudaStream_t s, int *per_sm) {
  auto kern = batch_queue_kernel<S, EOS>;
  if (per_sm) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, NTH, 0);
  void *args[] = {(void *)&boxes, (void *)&items, (void *)&nitems, (void *)&parity,
                  (void *)&done,  (void *)&ndone, (void *)&err};
  return cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(TXP, kRows), args, 0, s);
}

template <typename S>
cudaError_t batch_by_eos(int eos, const BatchBox *boxes, const int4 *items, int nitems, int parity, int grid,
                         int *done, int ndone, unsigned *err, cudaStream_t s, int *per_sm) {
  switch (eos) {
    case kEosCS: return batch_launch<S, kEosCS>(boxes, items, nitems, parity, grid, done, ndone, err, s, per_sm);
    case kEosExp: return batch_launch<S, kEosExp>(boxes, items, nitems, parity, grid, done, ndone, err, s, per_sm);
    default: return batch_launch<S, kEosNone>(boxes, items, nitems, parity, grid, done, ndone, err, s, per_sm);
  }
}

// Psi jobs go to the first free item at least `lag` items after the last of
// the fused jobs they read (ready[]); fused job j sits in item j.  Checks the
// result as the single-box list does.
bool place_psi_jobs(std::vector<int4> &out, const std::vector<long long> &ready, const std::vector<int2> &job,
                    long long nf, long long lag) {
  std::vector<long long> order((size_t)nf);
  for (long long p = 0; p < nf; ++p) order[p] = p;
  std::stable_sort(order.begin(), order.end(), [&](long long a, long long b) { return ready[a] < ready[b]; });
  long long next = 0;
  for (long long p : order) {
    const long long k = std::max(next, ready[p] + lag);
    while ((long long)out.size() <= k) out.push_back(make_int4(-1, -1, -1, -1));
    out[k].z = job[p].x;
    out[k].w = job[p].y;
    next = k + 1;
  }
  return (long long)out.size() < (1LL << 31);
}

}  // namespace

bool queue_supported(const KParams &P, int precision) { return precision != kF64 && P.nx % 2 == 0; }

cudaError_t queue_grid(int precision, int *grid) {
  int per_sm = 0, dev = 0, sms = 0;
  cudaError_t e = precision == kF32 ? occupancy_of<float>(&per_sm) : occupancy_of<__half>(&per_sm);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  *grid = per_sm * sms;
  return cudaSuccess;
}

size_t queue_counters(const KParams &P) { return (size_t)P.nz * tile_geo(P).T + 32; }  // + the claim counter

bool queue_items(const KParams &P, int grid, std::vector<int4> &out) {
  const TileGeo G = tile_geo(P);
  const long long nf = (long long)P.nz * G.T;
  if (P.nz < 3 || grid < 1 || nf >= (1LL << 30)) return false;
  // fused job j = (j / T, j % T); psi job (z, t) is ready after the last of the
  // 27 fused jobs it reads and goes to the first free item >= ready + lag, half
  // a wave of the grid later (at least one item)
  const long long lag = std::max(1, grid / 2);
  std::vector<long long> ready((size_t)nf);
  for (long long p = 0; p < nf; ++p) {
    const int z = (int)(p / G.T), t = (int)(p % G.T), tx = t % G.ntx, ty = t / G.ntx;
    long long r = -1;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int zz = (z + dz + P.nz) % P.nz, yy = (ty + dy + G.nty) % G.nty, xx = (tx + dx + G.ntx) % G.ntx;
          r = std::max(r, (long long)zz * G.T + yy * G.ntx + xx);
        }
    ready[p] = r;
  }
  std::vector<long long> order((size_t)nf);
  for (long long p = 0; p < nf; ++p) order[p] = p;
  std::stable_sort(order.begin(), order.end(), [&](long long a, long long b) { return ready[a] < ready[b]; });
  out.assign((size_t)nf, make_int4(-1, -1, -1, -1));
  for (long long j = 0; j < nf; ++j) out[j] = make_int4((int)(j / G.T), (int)(j % G.T), -1, -1);
  long long next = 0;  // first item that may still take a psi job
  for (long long p : order) {
    const long long k = std::max(next, ready[p] + lag);
    while ((long long)out.size() <= k) out.push_back(make_int4(-1, -1, -1, -1));
    out[k].z = (int)(p / G.T);
    out[k].w = (int)(p % G.T);
    next = k + 1;
  }
  if ((long long)out.size() >= (1LL << 31)) return false;
  // check: every job once; each psi job in an item after the fused jobs it reads
  std::vector<char> fseen((size_t)nf, 0), pseen((size_t)nf, 0);
  for (size_t k = 0; k < out.size(); ++k) {
    const int4 it = out[k];
    if (it.x >= 0) {
      const long long j = (long long)it.x * G.T + it.y;
      if (j != (long long)k || fseen[j]) return false;
      fseen[j] = 1;
    }
    if (it.z >= 0) {
      if (it.z >= P.nz || it.w < 0 || it.w >= G.T) return false;
      const long long p = (long long)it.z * G.T + it.w;
      if (pseen[p] || ready[p] >= (long long)k) return false;
      pseen[p] = 1;
    }
  }
  for (long long p = 0; p < nf; ++p)
    if (!fseen[p] || !pseen[p]) return false;
  return true;
}

cudaError_t launch_queue(const KParams &P, int precision, int op, bool sigma, bool df, const void *g_in, void *g_out,
                         const void *psi_in, void *psi_out, const QueueState &q, int stamp, unsigned *err,
                         cudaStream_t s) {
  if (!queue_supported(P, precision)) return cudaErrorInvalidValue;
  if (precision == kF32) return by_op<float>(P, op, sigma, df, g_in, g_out, psi_in, psi_out, q, stamp, err, s);
  return by_op<__half>(P, op, sigma, df, g_in, g_out, psi_in, psi_out, q, stamp, err, s);
}

int batch_tile_width(int nx) {
  // the widest of 64, 32, 16 with the fewest idle columns in the last tile
  int best = 64;
  long long waste = (long long)(nx + 63) / 64 * 64 - nx;
  for (int tw : {32, 16}) {
    const long long w = (long long)(nx + tw - 1) / tw * tw - nx;
    if (w < waste) best = tw, waste = w;
  }
  return best;
}

int batch_queue_tiles(const KParams &P) { return batch_geo(P, batch_tile_width(P.nx)).T; }

void batch_queue_geometry(BatchBox &d) {
  d.tw = batch_tile_width(d.P.nx);
  const BatchGeo G = batch_geo(d.P, d.tw);
  d.ntx = G.ntx;
  d.nty = G.nty;
  d.T = G.T;
  d.th = G.th;
  d.hshift = d.tw == 64 ? 5 : (d.tw == 32 ? 4 : 3);  // log2 of the node pairs across a tile
  d.ntx_m = ((1ull << 32) + (unsigned long long)G.ntx - 1) / (unsigned long long)G.ntx;
}

bool batch_queue_items(const std::vector<const KParams *> &boxes, int grid, std::vector<int4> &out,
                       std::vector<int> &base, long long *ncounters) {
  // fused jobs box by box, plane by plane: global fused position = item index
  std::vector<long long> first(boxes.size() + 1, 0);
  base.assign(boxes.size(), 0);
  for (size_t b = 0; b < boxes.size(); ++b) {
    const KParams &P = *boxes[b];
    const BatchGeo G = batch_geo(P, batch_tile_width(P.nx));
    if (P.nz < 3 || P.nx % 2 != 0 || P.nz > 0xffff || G.T > 0xffff || grid < 1) return false;
    first[b + 1] = first[b] + (long long)P.nz * G.T;
    if (first[b + 1] >= (1LL << 30)) return false;
    base[b] = (int)first[b];
  }
  const long long nf = first.back();
  *ncounters = nf;
  out.assign((size_t)nf, make_int4(-1, -1, -1, -1));
  std::vector<long long> ready((size_t)nf);
  std::vector<int2> job((size_t)nf);  // (box, z | tile << 16) of psi job p (same numbering as fused job p)
  for (size_t b = 0; b < boxes.size(); ++b) {
    const KParams &P = *boxes[b];
    const BatchGeo G = batch_geo(P, batch_tile_width(P.nx));
    for (int z = 0; z < P.nz; ++z)
      for (int t = 0; t < G.T; ++t) {
        const long long j = first[b] + (long long)z * G.T + t;
        const int zt = (int)((unsigned)z | ((unsigned)t << 16));
        out[j] = make_int4((int)b, zt, -1, -1);
        job[j] = make_int2((int)b, zt);
        const int tx = t % G.ntx, ty = t / G.ntx;
        long long r = -1;
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              const int zz = (z + dz + P.nz) % P.nz, yy = (ty + dy + G.nty) % G.nty, xx = (tx + dx + G.ntx) % G.ntx;
              r = std::max(r, first[b] + (long long)zz * G.T + yy * G.ntx + xx);
            }
        ready[j] = r;
      }
  }
  if (!place_psi_jobs(out, ready, job, nf, std::max(1, grid / 2))) return false;
  // check: every job once, each psi job in an item after the fused jobs it reads
  std::vector<char> fseen((size_t)nf, 0), pseen((size_t)nf, 0);
  for (size_t k = 0; k < out.size(); ++k) {
    const int4 it = out[k];
    for (int side = 0; side < 2; ++side) {
      const int b = side ? it.z : it.x;
      if (b < 0) continue;
      if (b >= (int)boxes.size()) return false;
      const unsigned zt = (unsigned)(side ? it.w : it.y);
      const int z = (int)(zt & 0xffffu), t = (int)(zt >> 16);
      const BatchGeo G = batch_geo(*boxes[b], batch_tile_width(boxes[b]->nx));
      if (z >= boxes[b]->nz || t >= G.T) return false;
      const long long j = first[b] + (long long)z * G.T + t;
      if (!side) {
        if (j != (long long)k || fseen[j]) return false;
        fseen[j] = 1;
      } else {
        if (pseen[j] || ready[j] >= (long long)k) return false;
        pseen[j] = 1;
      }
    }
  }
  for (long long p = 0; p < nf; ++p)
    if (!fseen[p] || !pseen[p]) return false;
  return true;
}

cudaError_t batch_queue_grid(int precision, int eos, int *grid) {
  int per_sm = 0, dev = 0, sms = 0;
  cudaError_t e = precision == kF32
                      ? batch_by_eos<float>(eos, nullptr, nullptr, 0, 0, 0, nullptr, 0, nullptr, 0, &per_sm)
                      : batch_by_eos<__half>(eos, nullptr, nullptr, 0, 0, 0, nullptr, 0, nullptr, 0, &per_sm);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  *grid = per_sm * sms;
  return cudaSuccess;
}

cudaError_t launch_batch_queue(int precision, int eos, const BatchBox *boxes, const int4 *items, int nitems,
                               int parity, int grid, int *done, int ndone, unsigned *err, cudaStream_t s) {
  if (precision == kF32)
    return batch_by_eos<float>(eos, boxes, items, nitems, parity, grid, done, ndone, err, s, nullptr);
  if (precision == kF16)
    return batch_by_eos<__half>(eos, boxes, items, nitems, parity, grid, done, ndone, err, s, nullptr);
  return cudaErrorInvalidValue;
}

}  // namespace lbm
