// Two-pass kernels for the FP32-arithmetic forms with two x-adjacent nodes per
// thread (Nx even).
//
// A thread owns the pair (x, x+1), x even.  Populations that arrive along
// e_x = 0 come from an aligned pair (x, x+1) of the source row: one 64-bit
// load (FP32 storage) or 32-bit load (FP16 storage).  Those with e_x = +1 come
// from (x-1, x) and those with e_x = -1 from (x+1, x+2), read as two scalars.
// The psi neighbourhood is read the same way: the nine rows of the stencil as
// aligned pairs plus x-1 and x+2 where a direction moves in x.  All arithmetic
// of the two nodes runs on packed FP32 pairs (V2): per node it is the
// arithmetic of the one-node kernels in lbm_kernels.cu, and a packed
// instruction issues the work of two nodes.
#include <cuda_fp16.h>

#include <algorithm>

#include "lbm_device.cuh"
#include "lbm_internal.h"
#include "lbm_pair.cuh"
#include "lbm_pair15.cuh"
#include "lbm_q15.cuh"

namespace lbm {
namespace {

// psi(x + e_a) of both nodes, p[a] (Eq. 15 stencil).
__device__ __forceinline__ void gather_psi_pair(const float *__restrict__ psi, const Nbhd &nb, const PairX &px,
                                                V2 p[19]) {
  // a row with x-moving directions: centre pair, x - 1 and x + 2
  auto row3 = [&](int row, V2 &c, V2 &plus, V2 &minus) {
    const float2 m = __ldg((const float2 *)(psi + row + px.x));
    const float l = __ldg(psi + row + px.xm1), r = __ldg(psi + row + px.xp2);
    c = V2(m);
    plus = V2(m.y, r);   // psi(x + 1), psi(x + 2)
    minus = V2(l, m.x);  // psi(x - 1), psi(x)
  };
  auto row1 = [&](int row) { return V2(__ldg((const float2 *)(psi + row + px.x))); };
  row3(nb.r00, p[0], p[1], p[2]);
  row3(nb.rp0, p[3], p[7], p[10]);
  row3(nb.rm0, p[4], p[9], p[8]);
  row3(nb.r0p, p[5], p[11], p[14]);
  row3(nb.r0m, p[6], p[13], p[12]);
  p[15] = row1(nb.rpp);
  p[16] = row1(nb.rmm);
  p[17] = row1(nb.rpm);
  p[18] = row1(nb.rmp);
}

__device__ __forceinline__ bool pair_of_thread(const KParams &P, PairX &px, int &y, int &z) {
  const int x = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  y = blockIdx.y * blockDim.y + threadIdx.y;
  z = blockIdx.z;
  if (x >= P.nx || y >= P.ny) return false;
  px.x = x;
  px.xm1 = x == 0 ? P.nx - 1 : x - 1;
  px.xp2 = x + 2 >= P.nx ? x + 2 - P.nx : x + 2;
  return true;
}

template <typename S, int EOS, bool DF>
__global__ void __launch_bounds__(128) psi_pair_kernel(const S *__restrict__ g, float *__restrict__ psi,
                                                       const KParams P, unsigned *__restrict__ err) {
  PairX px;
  int y, z;
  if (!pair_of_thread(P, px, y, z)) return;
  const Nbhd nb(px.x, y, z, P);
  V2 f[19];
  pull_pair<S>(g, (unsigned)P.n, nb, px, f);
  unsigned e = 0;
  *(float2 *)(psi + nb.self) = psi_pair<EOS, DF>(drho_pair(f), P, e);
  if (e) atomicOr(err, e);
}

template <typename S, int OP, bool SIGMA>
__global__ void __launch_bounds__(128) fused_pair_kernel(const S *__restrict__ g_in, S *__restrict__ g_out,
                                                         const float *__restrict__ psi, const KParams P) {
  PairX px;
  int y, z;
  if (!pair_of_thread(P, px, y, z)) return;
  const Nbhd nb(px.x, y, z, P);
  V2 f[19];
  pull_pair<S>(g_in, (unsigned)P.n, nb, px, f);
  V2 p[19];
  gather_psi_pair(psi, nb, px, p);
  force_collide_pair<OP, SIGMA>(f, p, P, Rates<V2>(P), OP);
#pragma unroll
  for (int a = 0; a < 19; ++a) PairIO<S>::st2(g_out + (size_t)a * P.n + nb.self, a, f[a]);
}

// ------------------------------------------------------------------ D3Q15
// The same two-node scheme for the D3Q15 variant (lbm_pair15.cuh).

template <typename S, int EOS, bool DF>
__global__ void __launch_bounds__(128) psi_pair15_kernel(const S *__restrict__ g, float *__restrict__ psi,
                                                         const KParams P, unsigned *__restrict__ err) {
  PairX px;
  int y, z;
  if (!pair_of_thread(P, px, y, z)) return;
  const Nbhd nb(px.x, y, z, P);
  V2 f[q15::kQ];
  pull_pair15<S>(g, (unsigned)P.n, nb, px, f);
  unsigned e = 0;
  *(float2 *)(psi + nb.self) = psi_pair<EOS, DF>(q15::drho(f), P, e);
  if (e) atomicOr(err, e);
}

template <typename S, bool SIGMA>
__global__ void __launch_bounds__(128) fused_pair15_kernel(const S *__restrict__ g_in, S *__restrict__ g_out,
                                                           const float *__restrict__ psi, const KParams P) {
  PairX px;
  int y, z;
  if (!pair_of_thread(P, px, y, z)) return;
  fused_pair15_at<S, SIGMA>(g_in, g_out, psi, P, px.x, y, z);
}

dim3 pair_grid(const KParams &P, const Launch &L) {
  return dim3((P.nx / 2 + 31) / 32, (P.ny + L.by - 1) / L.by, P.nz);
}

template <typename S, bool DF>
cudaError_t psi_pair_dispatch(const KParams &P, const void *g, void *psi, unsigned *err, const Launch &L) {
  const dim3 grid = pair_grid(P, L), block(32, L.by);
  const S *gg = (const S *)g;
  float *pp = (float *)psi;
  if (P.q == 15) {
    switch (P.eos) {
      case kEosCS: psi_pair15_kernel<S, kEosCS, DF><<<grid, block, 0, L.stream>>>(gg, pp, P, err); break;
      case kEosExp: psi_pair15_kernel<S, kEosExp, DF><<<grid, block, 0, L.stream>>>(gg, pp, P, err); break;
      default: psi_pair15_kernel<S, kEosNone, false><<<grid, block, 0, L.stream>>>(gg, pp, P, err); break;
    }
    return cudaGetLastError();
  }
  switch (P.eos) {
    case kEosCS: psi_pair_kernel<S, kEosCS, DF><<<grid, block, 0, L.stream>>>(gg, pp, P, err); break;
    case kEosExp: psi_pair_kernel<S, kEosExp, DF><<<grid, block, 0, L.stream>>>(gg, pp, P, err); break;
    default: psi_pair_kernel<S, kEosNone, false><<<grid, block, 0, L.stream>>>(gg, pp, P, err); break;
  }
  return cudaGetLastError();
}

template <typename S>
cudaError_t fused_pair_dispatch(const KParams &P, int op, bool sigma, const void *g_in, void *g_out,
                                const void *psi, const Launch &L) {
  const dim3 grid = pair_grid(P, L), block(32, L.by);
  const S *gi = (const S *)g_in;
  S *go = (S *)g_out;
  const float *pp = (const float *)psi;
  if (P.q == 15) {
    if (sigma) fused_pair15_kernel<S, true><<<grid, block, 0, L.stream>>>(gi, go, pp, P);
    else fused_pair15_kernel<S, false><<<grid, block, 0, L.stream>>>(gi, go, pp, P);
  } else if (op == kNonOrth) {
    if (sigma) fused_pair_kernel<S, kNonOrth, true><<<grid, block, 0, L.stream>>>(gi, go, pp, P);
    else fused_pair_kernel<S, kNonOrth, false><<<grid, block, 0, L.stream>>>(gi, go, pp, P);
  } else {
    if (sigma) fused_pair_kernel<S, kOrth, true><<<grid, block, 0, L.stream>>>(gi, go, pp, P);
    else fused_pair_kernel<S, kOrth, false><<<grid, block, 0, L.stream>>>(gi, go, pp, P);
  }
  return cudaGetLastError();
}

// Batched boxes, two-pass step, psi pass: work item w = (box, tile_x | tile_y
// << 16, z0, z1) is a TXP x TY tile of pairs (2 TXP x TY nodes) of one box
// through planes [z0, z1).  The fused pass (batch_flat_fused_kernel) reads
// level in = cur ^ parity (populations and psi) and writes the populations of
// level in ^ 1; this pass then evaluates psi of level in ^ 1, so after a step
// psi of the current level is always valid.  (A flat grid of one plane per
// block, as for the fused pass, measured 2 % slower here.)
template <typename S, int EOS, int TXP, int TY>
__global__ void __launch_bounds__(TXP *TY) batch_psi_kernel(const BatchBox *__restrict__ boxes,
                                                            const int4 *__restrict__ items, int nitems, int parity,
                                                            unsigned *__restrict__ err) {
  __shared__ BatchBox bb;
  const int tid = threadIdx.y * TXP + threadIdx.x;
  unsigned e = 0;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int4 w = items[it];
    __syncthreads();  // every thread is done with the previous item's descriptor
    {
      const int *src = (const int *)(boxes + w.x);
      int *dst = (int *)&bb;
      for (int k = tid; k < (int)(sizeof(BatchBox) / sizeof(int)); k += TXP * TY) dst[k] = src[k];
    }
    __syncthreads();
    const KParams &P = bb.P;
    const int in = bb.cur ^ parity;
    const int x = (w.y & 0xffff) * (2 * TXP) + 2 * threadIdx.x, y = (w.y >> 16) * TY + threadIdx.y;
    if (x >= P.nx || y >= P.ny) continue;
    const PairX px{x, x == 0 ? P.nx - 1 : x - 1, x + 2 >= P.nx ? x + 2 - P.nx : x + 2};
    const S *g = (const S *)bb.g[in ^ 1];
    float *psi = bb.psi[in ^ 1];
    for (int z = w.z; z < w.w; ++z) {
      const Nbhd nb(x, y, z, P);
      V2 f[19];
      pull_pair<S>(g, (unsigned)P.n, nb, px, f);
      *(float2 *)(psi + nb.self) = psi_pair<EOS, false>(drho_pair(f), P, e);
    }
  }
  if (e) atomicOr(err, e);
}

// Threads per SM the flat fused kernel's registers are set for: 640 (at most 102 registers a thread; both
// operators fit without spilling, the orthogonal one took 108 unbounded; 80 registers spilled and was slower).
constexpr int kFlatFusedThreadsPerSM = 640;

// The fused pass of a batch as a flat grid, one launch per operator: block b
// is one plane of one 2 TXP x TY tile of one box, block_box[offset + b] names
// the box, whose first block is its descriptor's qbase; planes are numbered
// box by box, tiles x-fastest within a plane.  One node pair per thread and no
// loop, as in fused_pair_kernel: a persistent kernel looping over the planes of
// an item held 128 registers (16 warps per SM) and reached 0.86 of the copy
// bandwidth, this one holds 96 (5 blocks of 128 threads) and 0.94.
template <typename S, int OP, int TXP, int TY>
__global__ void __launch_bounds__(TXP *TY, kFlatFusedThreadsPerSM / (TXP * TY)) batch_flat_fused_kernel(const BatchBox *__restrict__ boxes,
                                                                   const int *__restrict__ block_box, int offset,
                                                                   int parity) {
  const int gb = offset + (int)blockIdx.x;
  const int slot = __ldg(block_box + gb);
  const BatchBox &bb = boxes[slot];  // read where used (cached; a copy to shared memory measured the same)
  const KParams &P = bb.P;
  const int ntx = (P.nx + 2 * TXP - 1) / (2 * TXP), nty = (P.ny + TY - 1) / TY, T = ntx * nty;
  const int local = gb - bb.qbase, z = local / T, t = local - z * T;
  const int x = (t % ntx) * (2 * TXP) + 2 * threadIdx.x, y = (t / ntx) * TY + threadIdx.y;
  if (x >= P.nx || y >= P.ny || z >= P.nz) return;
  const int in = bb.cur ^ parity;
  fused_pair_at<S, OP, true, false>((const S *)bb.g[in], (S *)bb.g[in ^ 1], bb.psi[in], P, x, y, z, Rates<V2>(P));
}

// The fused and psi kernels of one step for a storage type and tile shape;
// with query set, per_sm receives their resident blocks per SM instead.
template <typename S, int TXP, int TY>
cudaError_t batch_pair_shape(int eos, const BatchBox *boxes, const int4 *items, int nitems, const int *block_box,
                             const int fused_blocks[2], int parity, int sms, int per_sm[2], bool query, unsigned *err,
                             cudaStream_t s) {
  using K = void (*)(const BatchBox *, const int4 *, int, int, unsigned *);
  K kpsi;
  switch (eos) {
    case kEosCS: kpsi = batch_psi_kernel<S, kEosCS, TXP, TY>; break;
    case kEosExp: kpsi = batch_psi_kernel<S, kEosExp, TXP, TY>; break;
    default: kpsi = batch_psi_kernel<S, kEosNone, TXP, TY>; break;
  }
  if (query) {
    per_sm[0] = 0;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[1], kpsi, TXP * TY, 0);
  }
  // fused pass: the flat launches (non-orthogonal boxes' blocks first in block_box, then the orthogonal ones)
  if (fused_blocks[0] > 0)
    batch_flat_fused_kernel<S, kNonOrth, TXP, TY><<<fused_blocks[0], dim3(TXP, TY), 0, s>>>(boxes, block_box, 0, parity);
  if (fused_blocks[1] > 0)
    batch_flat_fused_kernel<S, kOrth, TXP, TY><<<fused_blocks[1], dim3(TXP, TY), 0, s>>>(boxes, block_box, fused_blocks[0],
                                                                                       parity);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int grid = std::max(1, std::min(sms * std::max(per_sm[1], 1), nitems));
  kpsi<<<grid, dim3(TXP, TY), 0, s>>>(boxes, items, nitems, parity, err);
  return cudaGetLastError();
}

template <typename S>
cudaError_t batch_pair_tile(int tile, int eos, const BatchBox *boxes, const int4 *items, int nitems,
                            const int *block_box, const int fused_blocks[2], int parity, int sms, int per_sm[2],
                            bool query, unsigned *err, cudaStream_t s) {
  switch (tile) {
    case kTile32x4:
      return batch_pair_shape<S, 16, 4>(eos, boxes, items, nitems, block_box, fused_blocks, parity, sms, per_sm, query,
                                        err, s);
    case kTile64x4:
      return batch_pair_shape<S, 32, 4>(eos, boxes, items, nitems, block_box, fused_blocks, parity, sms, per_sm, query,
                                        err, s);
    default:
      return batch_pair_shape<S, 16, 8>(eos, boxes, items, nitems, block_box, fused_blocks, parity, sms, per_sm, query,
                                        err, s);
  }
}

cudaError_t batch_pair_dispatch(int precision, int tile, int eos, const BatchBox *boxes, const int4 *items, int nitems,
                                const int *block_box, const int fused_blocks[2], int parity, int sms, int per_sm[2],
                                bool query, unsigned *err, cudaStream_t s) {
  if (precision == kF32)
    return batch_pair_tile<float>(tile, eos, boxes, items, nitems, block_box, fused_blocks, parity, sms, per_sm, query,
                                  err, s);
  if (precision == kF16)
    return batch_pair_tile<__half>(tile, eos, boxes, items, nitems, block_box, fused_blocks, parity, sms, per_sm,
                                   query, err, s);
  return cudaErrorInvalidValue;
}

}  // namespace

bool pair_supported(const KParams &P, int precision) { return precision != kF64 && P.nx % 2 == 0; }

cudaError_t batch_pair_occupancy(int precision, int eos, int tile, int per_sm[2]) {
  const int none[2] = {0, 0};
  return batch_pair_dispatch(precision, tile, eos, nullptr, nullptr, 0, nullptr, none, 0, 0, per_sm, true, nullptr, 0);
}

cudaError_t launch_batch_pair(int precision, int eos, int tile, const BatchBox *boxes, const int4 *items, int nitems,
                              const int *block_box, const int fused_blocks[2], int parity, int sms,
                              const int per_sm[2], unsigned *err, cudaStream_t s) {
  int ps[2] = {per_sm[0], per_sm[1]};
  return batch_pair_dispatch(precision, tile, eos, boxes, items, nitems, block_box, fused_blocks, parity, sms, ps,
                             false, err, s);
}

cudaError_t launch_psi_pair(const KParams &P, int precision, const void *g, void *psi, unsigned *err,
                            const Launch &L, bool df) {
  if (precision == kF32)
    return df ? psi_pair_dispatch<float, true>(P, g, psi, err, L) : psi_pair_dispatch<float, false>(P, g, psi, err, L);
  return df ? psi_pair_dispatch<__half, true>(P, g, psi, err, L) : psi_pair_dispatch<__half, false>(P, g, psi, err, L);
}

cudaError_t launch_fused_pair(const KParams &P, int precision, int op, bool sigma, const void *g_in, void *g_out,
                              const void *psi, const Launch &L) {
  if (precision == kF32) return fused_pair_dispatch<float>(P, op, sigma, g_in, g_out, psi, L);
  return fused_pair_dispatch<__half>(P, op, sigma, g_in, g_out, psi, L);
}

}  // namespace lbm
