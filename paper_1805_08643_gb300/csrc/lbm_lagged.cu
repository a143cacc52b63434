// Single-pass time step for the FP32-arithmetic forms (Nx even) in which the
// psi pass of the next step trails the fused pass by one plane inside one
// persistent launch.
//
// psi(t+1) of plane z needs the post-collision populations of planes z-1, z,
// z+1 (Eqs. 5, 6), i.e. the fused pass of those planes by the blocks of the
// neighbouring tiles.  Every block owns x-y tiles of 64 x 4 nodes and marches
// z upwards: fused pass of plane z (as fused_pair_kernel: reads f(t) and
// psi(t), writes f*(t)), publishes "plane z of this tile done" in a flag, then,
// once the eight neighbouring tiles have published plane z-1 as well, evaluates
// psi(t+1) of plane z-2 (as psi_pair_kernel) from the populations just written,
// which are still in L2.  The planes whose stencils reach into the next or
// previous z chunk (or wrap) come last.
// DRAM traffic per node: f(t) read and f*(t) written once, psi(t) read and
// psi(t+1) written once (2 x 19 x s + 8 bytes) against 3 x 19 x s + 8 for the
// two launches; the arithmetic and its order are those of the two-pass step,
// so the results are equal bit for bit.
//
// Blocks wait on each other, so they must all be resident: the launch is
// cooperative (it fails instead of running if the grid does not fit), every
// wait is bounded (a wait that gives up sets kErrTimeout and goes on), and a
// flag holds the number of the launch that wrote it, so flags need no reset.
#include <cuda_fp16.h>

#include "lbm_device.cuh"
#include "lbm_internal.h"
#include "lbm_pair.cuh"

namespace lbm {
namespace {

constexpr int TXP = 32, TYR = 4;  // pair columns and rows per tile: 64 x 4 nodes
constexpr int NTH = TXP * TYR;

struct Tiles {
  int nx_t, ny_t, n;  // tiles in x, in y, total
};

__device__ __forceinline__ Tiles tiles_of(const KParams &P) {
  Tiles t;
  t.nx_t = (P.nx + 2 * TXP - 1) / (2 * TXP);
  t.ny_t = (P.ny + TYR - 1) / TYR;
  t.n = t.nx_t * t.ny_t;
  return t;
}

__device__ __forceinline__ int load_flag(const int *f) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
  return v;
}
__device__ __forceinline__ void store_flag(int *f, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(f), "r"(v) : "memory");
}

// Wait until the tiles around tile t (and t) have published plane z of launch
// `stamp` (plus P.wait_bias): thread k < 9 watches neighbour k, at most
// P.spin_limit polls; then the block synchronises.
__device__ __forceinline__ bool wait_neighbours(const int *flags, const Tiles &T, int t, int z, int nz, int stamp,
                                                const KParams &P) {
  bool ok = true;
  const int k = threadIdx.y * TXP + threadIdx.x;
  if (k < 9) {
    const int tx = t % T.nx_t, ty = t / T.nx_t;
    const int nxt = (tx + (k % 3) - 1 + T.nx_t) % T.nx_t, nyt = (ty + (k / 3) - 1 + T.ny_t) % T.ny_t;
    const int *f = flags + (size_t)(nyt * T.nx_t + nxt) * nz + z;
    const int target = stamp + P.wait_bias;
    int it = 0;
    while (load_flag(f) < target) {
      if (++it > P.spin_limit) {
        ok = false;
        break;
      }
      __nanosleep(64);
    }
  }
  return __syncthreads_and(ok);
}

template <typename S, int OP, bool SIGMA>
__device__ __forceinline__ void fused_plane(const S *__restrict__ g_in, S *__restrict__ g_out,
                                            const float *__restrict__ psi, const KParams &P, const Tiles &T, int t,
                                            int z, const Rates<V2> &r) {
  const int x = (t % T.nx_t) * 2 * TXP + 2 * threadIdx.x, y = (t / T.nx_t) * TYR + threadIdx.y;
  if (x >= P.nx || y >= P.ny) return;
  fused_pair_at<S, OP, SIGMA>(g_in, g_out, psi, P, x, y, z, r);
}

template <typename S, int EOS, bool DF>
__device__ __forceinline__ void psi_plane(const S *__restrict__ g, float *__restrict__ psi, const KParams &P,
                                          const Tiles &T, int t, int z, unsigned &e) {
  const int x = (t % T.nx_t) * 2 * TXP + 2 * threadIdx.x, y = (t / T.nx_t) * TYR + threadIdx.y;
  if (x >= P.nx || y >= P.ny) return;
  psi_pair_at_l2<S, EOS, DF>(g, psi, P, x, y, z, e);
}

// Block b works on z chunk b / per_chunk ([z0, z1), at least three planes) and
// on tiles b % per_chunk, + per_chunk, ... of it.
template <typename S, int OP, bool SIGMA, int EOS, bool DF>
__global__ void __launch_bounds__(NTH, 7) lagged_kernel(const S *__restrict__ g_in, S *__restrict__ g_out,
                                                     const float *__restrict__ psi_in, float *__restrict__ psi_out,
                                                     const KParams P, int zc, int per_chunk,
                                                     int *__restrict__ flags, int stamp, unsigned *__restrict__ err) {
  const Tiles T = tiles_of(P);
  const int nz = P.nz;
  const int chunk = blockIdx.x / per_chunk, t0 = blockIdx.x % per_chunk;
  const int z0 = chunk * zc, z1 = min(z0 + zc, nz);
  const Rates<V2> r(P);
  unsigned e = 0;
  const int tid = threadIdx.y * TXP + threadIdx.x;
  auto publish = [&](int z) {
    __threadfence();
    __syncthreads();
    if (tid == 0)
      for (int t = t0; t < T.n; t += per_chunk) store_flag(flags + (size_t)t * nz + z, stamp);
  };
  auto psi_of = [&](int z, int z_wait) {  // psi(t+1) of plane z once the neighbours have done plane z_wait
    for (int t = t0; t < T.n; t += per_chunk) {
      if (!wait_neighbours(flags, T, t, z_wait, nz, stamp, P)) e |= kErrTimeout;
      psi_plane<S, EOS, DF>(g_out, psi_out, P, T, t, z, e);
    }
  };
  for (int z = z0; z < z1; ++z) {
    for (int t = t0; t < T.n; t += per_chunk) fused_plane<S, OP, SIGMA>(g_in, g_out, psi_in, P, T, t, z, r);
    publish(z);
    // psi two planes behind: its last source plane z - 1 was published a plane
    // ago, so the neighbours are normally there already
    if (z >= z0 + 3) psi_of(z - 2, z - 1);
  }
  // z1 - 2; then the planes whose stencils reach into the neighbouring chunks
  // (or wrap): z1 - 1 needs plane z1 (first of the next chunk, done early), z0
  // needs plane z0 - 1 (last of the previous chunk, done at its end)
  psi_of(z1 - 2, z1 - 1);
  psi_of(z1 - 1, z1 == nz ? 0 : z1);
  psi_of(z0, z0 == 0 ? nz - 1 : z0 - 1);
  if (e) atomicOr(err, e);
}

template <typename S, int OP, bool SIGMA, int EOS, bool DF>
cudaError_t launch_kernel(const KParams &P, const void *g_in, void *g_out, const void *psi_in, void *psi_out,
                          int *flags, int stamp, unsigned *err, cudaStream_t s) {
  auto kern = lagged_kernel<S, OP, SIGMA, EOS, DF>;
  static int per_sm = 0, sms = 0;  // per process: one device
  if (per_sm == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NTH, 0);
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
  }
  // every block must be resident: as many z chunks (of at least three planes) as
  // the resident blocks cover the tiles; beyond one chunk, blocks own tiles in turn
  const int tiles = ((P.nx + 2 * TXP - 1) / (2 * TXP)) * ((P.ny + TYR - 1) / TYR);
  const int cap = per_sm * sms;
  int chunks = cap / tiles;
  if (chunks > P.nz / 3) chunks = P.nz / 3;
  if (chunks < 1) chunks = 1;
  int zc = (P.nz + chunks - 1) / chunks;
  while (chunks > 1 && P.nz - (chunks - 1) * zc < 3) zc = (P.nz + --chunks - 1) / chunks;
  chunks = (P.nz + zc - 1) / zc;
  const int per_block = chunks > 1 ? 1 : (tiles + cap - 1) / cap;  // tiles each block owns
  const int per_chunk = (tiles + per_block - 1) / per_block;       // blocks per chunk
  const int grid = per_chunk * chunks;
  const S *gi = (const S *)g_in;
  S *go = (S *)g_out;
  const float *pi = (const float *)psi_in;
  float *po = (float *)psi_out;
  KParams Pc = P;
  void *args[] = {(void *)&gi, (void *)&go,        (void *)&pi,    (void *)&po,    (void *)&Pc,
                  (void *)&zc, (void *)&per_chunk, (void *)&flags, (void *)&stamp, (void *)&err};
  return cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(TXP, TYR), args, 0, s);
}

template <typename S, int OP, bool SIGMA>
cudaError_t by_eos(const KParams &P, bool df, const void *g_in, void *g_out, const void *psi_in, void *psi_out,
                   int *flags, int stamp, unsigned *err, cudaStream_t s) {
  switch (P.eos) {
    case kEosCS:
      return df ? launch_kernel<S, OP, SIGMA, kEosCS, true>(P, g_in, g_out, psi_in, psi_out, flags, stamp, err, s)
                : launch_kernel<S, OP, SIGMA, kEosCS, false>(P, g_in, g_out, psi_in, psi_out, flags, stamp, err, s);
    case kEosExp:
      return df ? launch_kernel<S, OP, SIGMA, kEosExp, true>(P, g_in, g_out, psi_in, psi_out, flags, stamp, err, s)
                : launch_kernel<S, OP, SIGMA, kEosExp, false>(P, g_in, g_out, psi_in, psi_out, flags, stamp, err, s);
    default:
      return launch_kernel<S, OP, SIGMA, kEosNone, false>(P, g_in, g_out, psi_in, psi_out, flags, stamp, err, s);
  }
}

template <typename S>
cudaError_t by_op(const KParams &P, int op, bool sigma, bool df, const void *g_in, void *g_out, const void *psi_in,
                  void *psi_out, int *flags, int stamp, unsigned *err, cudaStream_t s) {
  if (op == kNonOrth)
    return sigma ? by_eos<S, kNonOrth, true>(P, df, g_in, g_out, psi_in, psi_out, flags, stamp, err, s)
                 : by_eos<S, kNonOrth, false>(P, df, g_in, g_out, psi_in, psi_out, flags, stamp, err, s);
  return sigma ? by_eos<S, kOrth, true>(P, df, g_in, g_out, psi_in, psi_out, flags, stamp, err, s)
               : by_eos<S, kOrth, false>(P, df, g_in, g_out, psi_in, psi_out, flags, stamp, err, s);
}

}  // namespace

bool lagged_supported(const KParams &P, int precision) { return precision != kF64 && P.nx % 2 == 0; }

size_t lagged_flag_count(const KParams &P) {
  return (size_t)((P.nx + 2 * TXP - 1) / (2 * TXP)) * ((P.ny + TYR - 1) / TYR) * P.nz;
}

cudaError_t launch_lagged(const KParams &P, int precision, int op, bool sigma, bool df, const void *g_in, void *g_out,
                          const void *psi_in, void *psi_out, int *flags, int stamp, unsigned *err, cudaStream_t s) {
  if (!lagged_supported(P, precision)) return cudaErrorInvalidValue;
  if (precision == kF32) return by_op<float>(P, op, sigma, df, g_in, g_out, psi_in, psi_out, flags, stamp, err, s);
  return by_op<__half>(P, op, sigma, df, g_in, g_out, psi_in, psi_out, flags, stamp, err, s);
}

}  // namespace lbm
