// Single-pass time step for the FP32-arithmetic forms (Nx even) that keeps psi
// on chip, with the work of a thread block split between producer and
// consumer warps.
//
// psi(t) of a node depends only on the populations pulled into it, rho(t) =
// sum_a f_a(x - e_a, t) (Eqs. 5, 6), so a block that owns an x-y tile of 32 x 8
// nodes can evaluate psi(t) for the tile and a one-node ring around it from the
// stored state, without psi of another block, and march the tile along z.
//  * Producer warps (4): for each plane, pull the populations of the tile's
//    128 node pairs and of the ring's 52 pairs (as lbm_kernels_pair.cu), put
//    the tile's into a shared staging buffer, sum rho, evaluate psi (Eq. 58
//    radicand in FP64) into a four-plane psi ring and signal the plane.  They
//    ask L2 for the plane after next and run up to two planes ahead of the
//    consumers (three staging buffers).
//  * Consumer warps (4): for plane z, once psi of plane z+1 is signalled, take
//    the staged populations of plane z and psi of planes z-1, z, z+1 from
//    shared memory, apply force and collision on packed FP32 pairs (as
//    lbm_kernels_pair.cu) and store f*; then release the plane.
// The consumers never wait on global memory and the producers never compute a
// collision; the hand-off is a set of mbarriers (one per psi slot, "full", and
// one per staging buffer, "empty"), every wait bounded.  DRAM traffic is one
// read and one write of the populations per step (the ring's reads hit L2,
// since the blocks of neighbouring tiles march the same planes at the same
// time); no psi array is read or written.
#include <cuda_fp16.h>

#include "lbm_async.cuh"
#include "lbm_device.cuh"
#include "lbm_internal.h"
#include "lbm_pair.cuh"

namespace lbm {
namespace {

constexpr int TX = 16, TY = 8;             // pair columns and rows: a 32 x 8 node tile
constexpr int BX = 2 * TX, BY = TY;
constexpr int NI = TX * TY;                // tile pairs = consumer threads
constexpr int NR = 2 * (TX + 2) + 2 * TY;  // ring pairs: two full rows (x = -2 .. BX), two side columns
constexpr int NPT = 128;                   // producer threads
constexpr int NTH = NI + NPT;
constexpr int PX = BX + 4, EY = BY + 2, NPSI = PX * EY;  // psi plane: local x -2 .. BX+1, y -1 .. BY
constexpr int NSTAGE = 3;                  // staging buffers of tile pairs
static_assert(NI == NPT && NR <= NPT, "each producer thread owns one tile pair and at most one ring pair");

// shared memory layout (bytes)
constexpr size_t kBarBytes = 64;                                    // full[4], empty[3]
constexpr size_t kPsiOff = kBarBytes;
constexpr size_t kStageOff = kPsiOff + (sizeof(float) * 4 * NPSI + 15) / 16 * 16;
constexpr size_t kRingOff = kStageOff + sizeof(float2) * NSTAGE * 19 * NI;  // end of the staging
constexpr size_t kSmemBytes = kRingOff;

__device__ __forceinline__ int wrapi(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// Ask L2 for the lines that the pull of pair (x, x+1), row y, plane z will read
// (one line per direction; the shifted neighbours x-1, x+2 share it or the next).
template <typename S>
__device__ __forceinline__ void prefetch_pair_l2(const S *__restrict__ g, const KParams &P, int x, int y, int z) {
  const Nbhd nb(x, y, z, P);
#pragma unroll
  for (int a = 0; a < 19; ++a)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(g + (size_t)a * P.n + src_row(nb, a) + x));
}

// Local coordinates of ring pair r: rows y = -1 and y = BY with x = -2 .. BX,
// then the side pairs x = -2 and x = BX of rows 0 .. BY-1.
__device__ __forceinline__ void ring_pair(int r, int &lx, int &ly) {
  if (r < 2 * (TX + 2)) {
    ly = r < TX + 2 ? -1 : BY;
    lx = 2 * (r % (TX + 2)) - 2;
  } else {
    const int k = r - 2 * (TX + 2);
    ly = k >> 1;
    lx = (k & 1) ? BX : -2;
  }
}

// Planes of a block are counted from z0 - 1: index m = z - z0 + 1.  psi of plane
// m lives in slot m & 3 (the (m >> 2)-th use of full[m & 3]); the staged tile
// pairs of plane m (decoded FP32 deviations) in buffer m % 3, released through
// empty[m % 3] once plane m is collided.
template <typename S, int OP, bool SIGMA, int EOS, bool DF>
__global__ void __launch_bounds__(NTH, 3)
    onchip_kernel(const S *__restrict__ g_in, S *__restrict__ g_out, const KParams P, int zc,
                  unsigned *__restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long *full = (unsigned long long *)smem;
  unsigned long long *empty = full + 4;
  float *psi = (float *)(smem + kPsiOff);
  float2 *stage = (float2 *)(smem + kStageOff);  // [NSTAGE][19][NI]
  const int tid = threadIdx.x;
  const int tiles_x = (P.nx + BX - 1) / BX, tiles = tiles_x * ((P.ny + BY - 1) / BY);
  const int t = blockIdx.x % tiles;
  const int x0 = (t % tiles_x) * BX, y0 = (t / tiles_x) * BY;
  const int z0 = (blockIdx.x / tiles) * zc, z1 = min(z0 + zc, P.nz);
  if (tid == 0) {
    for (int k = 0; k < 4; ++k) mbar_init(&full[k], NPT);
    for (int k = 0; k < 3; ++k) mbar_init(&empty[k], NI);
  }
  __syncthreads();
  unsigned e = 0;
  auto psi_slot = [&](int m) { return psi + (m & 3) * NPSI; };
  auto stage_buf = [&](int m) { return stage + (m % NSTAGE) * 19 * NI; };

  if (tid >= NI) {
    // ---------------------------------------------------------------- producer
    const int p = tid - NI;
    const int lxp = 2 * (p % TX), lyp = p / TX;
    const int gxp = wrapi(x0 + lxp, P.nx), gyp = wrapi(y0 + lyp, P.ny), cs = (lyp + 1) * PX + lxp + 2;
    const bool has_ring = p < NR;
    int rlx = 0, rly = 0;
    if (has_ring) ring_pair(p, rlx, rly);
    const int rgx = wrapi(x0 + rlx, P.nx), rgy = wrapi(y0 + rly, P.ny), cr = (rly + 1) * PX + rlx + 2;
    const PairX pxp{gxp, gxp == 0 ? P.nx - 1 : gxp - 1, gxp + 2 >= P.nx ? gxp + 2 - P.nx : gxp + 2};
    const PairX pxr{rgx, rgx == 0 ? P.nx - 1 : rgx - 1, rgx + 2 >= P.nx ? rgx + 2 - P.nx : rgx + 2};
    const int m_last = z1 - z0 + 1;  // planes z0 - 1 .. z1
    for (int m = 0; m <= m_last; ++m) {
      // staging buffer m % 3 last held plane m - 3 and psi slot m & 3 plane m - 4:
      // the collision of plane m - 3 is the last to read either, so wait for it
      // (the ((m - 4) / 3)-th release of buffer (m - 3) % 3)
      if (m >= 4 && !mbar_wait(&empty[(m - 3) % NSTAGE], ((m - 4) / NSTAGE) & 1, P.spin_limit)) {
        e |= kErrTimeout;
        break;
      }
      const int zw = wrapi(z0 - 1 + m, P.nz);
      if (m + 2 <= m_last) {  // ask L2 for the plane after next
        const int zn = wrapi(z0 + 1 + m, P.nz);
        prefetch_pair_l2<S>(g_in, P, gxp, gyp, zn);
        if (has_ring) prefetch_pair_l2<S>(g_in, P, rgx, rgy, zn);
      }
      float *ps = psi_slot(m);
      V2 f[19];
      pull_pair<S>(g_in, (unsigned)P.n, Nbhd(gxp, gyp, zw, P), pxp, f);
      float2 *st = stage_buf(m) + p;
#pragma unroll
      for (int a = 0; a < 19; ++a) st[a * NI] = f[a].v;
      *(float2 *)(ps + cs) = psi_pair<EOS, DF>(drho_pair(f), P, e);
      if (has_ring) {
        pull_pair<S>(g_in, (unsigned)P.n, Nbhd(rgx, rgy, zw, P), pxr, f);
        *(float2 *)(ps + cr) = psi_pair<EOS, DF>(drho_pair(f), P, e);
      }
      mbar_arrive(&full[m & 3]);
    }
  } else {
    // ---------------------------------------------------------------- consumer
    const int lx = 2 * (tid % TX), ly = tid / TX;
    const bool owned = x0 + lx < P.nx && y0 + ly < P.ny;
    const int gx = wrapi(x0 + lx, P.nx), gy = wrapi(y0 + ly, P.ny), c = (ly + 1) * PX + lx + 2;
    const Rates<V2> r(P);
    bool ok = mbar_wait(&full[0], 0, P.spin_limit) && mbar_wait(&full[1], 0, P.spin_limit);  // planes z0 - 1 and z0
    for (int z = z0; z < z1 && ok; ++z) {
      const int m = z - z0 + 1;
      if (!mbar_wait(&full[(m + 1) & 3], ((m + 1) >> 2) & 1, P.spin_limit)) {  // psi of plane z + 1
        ok = false;
        break;
      }
      if (owned) {
        V2 f[19];
        const float2 *st = stage_buf(m) + tid;
#pragma unroll
        for (int a = 0; a < 19; ++a) f[a] = V2(st[a * NI]);
        // p[a] = psi(x + e_a): rows (y + e_y, z + e_z) of the shared planes
        const float *pm = psi_slot(m - 1) + c, *p0 = psi_slot(m) + c, *pp = psi_slot(m + 1) + c;
        V2 q[19];
        auto row3 = [&](const float *s, V2 &ctr, V2 &plus, V2 &minus) {
          const float2 v = *(const float2 *)s;
          const float l = s[-1], rr = s[2];
          ctr = V2(v);
          plus = V2(v.y, rr);
          minus = V2(l, v.x);
        };
        row3(p0, q[0], q[1], q[2]);
        row3(p0 + PX, q[3], q[7], q[10]);
        row3(p0 - PX, q[4], q[9], q[8]);
        row3(pp, q[5], q[11], q[14]);
        row3(pm, q[6], q[13], q[12]);
        q[15] = V2(*(const float2 *)(pp + PX));
        q[16] = V2(*(const float2 *)(pm - PX));
        q[17] = V2(*(const float2 *)(pm + PX));
        q[18] = V2(*(const float2 *)(pp - PX));
        force_collide_pair<OP, SIGMA>(f, q, P, r, OP);
        const size_t self = ((size_t)z * P.ny + gy) * P.nx + gx;
#pragma unroll
        for (int a = 0; a < 19; ++a) PairIO<S>::st2(g_out + (size_t)a * P.n + self, a, f[a]);
      }
      mbar_arrive(&empty[m % NSTAGE]);
    }
    if (!ok) e |= kErrTimeout;
  }
  if (e) atomicOr(err, e);
}

template <typename S, int OP, bool SIGMA, int EOS, bool DF>
cudaError_t launch_kernel(const KParams &P, const void *g_in, void *g_out, unsigned *err, cudaStream_t s) {
  auto kern = onchip_kernel<S, OP, SIGMA, EOS, DF>;
  static int per_sm = 0, sms = 0;  // per process: one device
  if (per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NTH, kSmemBytes);
    if (e != cudaSuccess) return e;
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
  }
  // z chunk: the count of equal chunks that minimises (waves of blocks) x
  // (planes per chunk + the three planes of psi a block evaluates beyond them)
  const long long slots = (long long)per_sm * sms;
  const long long tiles = (long long)((P.nx + BX - 1) / BX) * ((P.ny + BY - 1) / BY);
  int zc = P.nz;
  long long best = -1;
  for (int chunks = 1; chunks <= (P.nz >= 16 ? P.nz / 8 : 1); ++chunks) {
    const int c = (P.nz + chunks - 1) / chunks;
    const long long blocks = tiles * ((P.nz + c - 1) / c);
    const long long cost = (blocks + slots - 1) / slots * (c + 3);
    if (best < 0 || cost < best) best = cost, zc = c;
  }
  const long long blocks = tiles * ((P.nz + zc - 1) / zc);
  kern<<<(unsigned)blocks, NTH, kSmemBytes, s>>>((const S *)g_in, (S *)g_out, P, zc, err);
  return cudaGetLastError();
}

template <typename S, int OP, bool SIGMA>
cudaError_t by_eos(const KParams &P, bool df, const void *g_in, void *g_out, unsigned *err, cudaStream_t s) {
  switch (P.eos) {
    case kEosCS:
      return df ? launch_kernel<S, OP, SIGMA, kEosCS, true>(P, g_in, g_out, err, s)
                : launch_kernel<S, OP, SIGMA, kEosCS, false>(P, g_in, g_out, err, s);
    case kEosExp:
      return df ? launch_kernel<S, OP, SIGMA, kEosExp, true>(P, g_in, g_out, err, s)
                : launch_kernel<S, OP, SIGMA, kEosExp, false>(P, g_in, g_out, err, s);
    default: return launch_kernel<S, OP, SIGMA, kEosNone, false>(P, g_in, g_out, err, s);
  }
}

template <typename S>
cudaError_t by_op(const KParams &P, int op, bool sigma, bool df, const void *g_in, void *g_out, unsigned *err,
                  cudaStream_t s) {
  if (op == kNonOrth)
    return sigma ? by_eos<S, kNonOrth, true>(P, df, g_in, g_out, err, s)
                 : by_eos<S, kNonOrth, false>(P, df, g_in, g_out, err, s);
  return sigma ? by_eos<S, kOrth, true>(P, df, g_in, g_out, err, s)
               : by_eos<S, kOrth, false>(P, df, g_in, g_out, err, s);
}

}  // namespace

bool onchip_supported(const KParams &P, int precision) { return precision != kF64 && P.nx % 2 == 0; }

cudaError_t launch_onchip(const KParams &P, int precision, int op, bool sigma, bool df, const void *g_in, void *g_out,
                          unsigned *err, cudaStream_t s) {
  if (!onchip_supported(P, precision)) return cudaErrorInvalidValue;
  if (precision == kF32) return by_op<float>(P, op, sigma, df, g_in, g_out, err, s);
  return by_op<__half>(P, op, sigma, df, g_in, g_out, err, s);
}

}  // namespace lbm
