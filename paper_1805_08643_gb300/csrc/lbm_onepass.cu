// Single-pass time step for the FP32-arithmetic forms: force + collision +
// pull streaming of step t and the psi of step t+1 in one kernel, so the
// populations are read once and written once per step (no separate psi pass).
//
// Each CTA owns an x-y tile of BX x BY nodes and marches along z through a
// chunk of planes.  psi(t+1)(x) needs rho(x, t+1) = sum_a f*_a(x - e_a, t):
// post-collision values of the neighbours.  The CTA therefore computes the
// collision on the tile plus a one-node ring in x and y (those results are not
// stored), and one extra plane below and above its chunk.  After the collision
// of plane z it stages the 18 moving f*_a of the extended plane in shared
// memory; each interior node gathers the contributions that stream into its
// own plane (e_z = 0), into plane z+1 (e_z = +1) and into plane z-1 (e_z = -1).
// rho(t+1) of plane z-1 is complete after plane z: the CTA then evaluates the
// EOS (FP64 polynomial, see eos_psi) and stores psi(t+1).  psi(t) is read
// from one buffer and psi(t+1) written to the other; no CTA waits for another.
#include <cuda_fp16.h>

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {
namespace {

template <int PREC> struct OneTypes;
template <> struct OneTypes<kF32> { using S = float; };
template <> struct OneTypes<kF16> { using S = __half; };

__device__ __forceinline__ int wrap(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// Shared memory of one CTA: two buffers of the 18 moving f* of an extended
// plane (the exchange is double-buffered so one barrier per plane suffices)
// and a ring of four psi(t) planes of (BX+4) x (BY+4) nodes.
template <int BX, int BY> struct OneSmem {
  static constexpr int EX = BX + 2, EY = BY + 2, NE = EX * EY;
  static constexpr int PX = BX + 4, PY = BY + 4, NP = PX * PY;
  static constexpr size_t bytes = sizeof(float) * (2 * 18 * NE + 4 * NP);
};

// resident CTAs per SM the register budget is sized for
template <int BX, int BY> constexpr int one_min_blocks() { return (BX + 2) * (BY + 2) <= 256 ? 4 : 2; }

// Operator chosen per thread block at run time (batched boxes of both kinds).
constexpr int kOpRuntime = 2;

// One x-y tile of one box marched through planes [z0, z1): the whole single
// pass for those nodes.  OP is kOrth, kNonOrth or kOpRuntime (then op_rt picks).
template <int PREC, int OP, bool SIGMA, int EOS, int BX, int BY>
__device__ __forceinline__ void onepass_tile(const typename OneTypes<PREC>::S *__restrict__ g_in,
                                             typename OneTypes<PREC>::S *__restrict__ g_out,
                                             const float *__restrict__ psi_in, float *__restrict__ psi_out,
                                             const KParams &P, int x0, int y0, int z0, int z1, int op_rt,
                                             unsigned &e, float *smem) {
  using S = typename OneTypes<PREC>::S;
  using SM = OneSmem<BX, BY>;
  constexpr int EX = SM::EX, NE = SM::NE, PX = SM::PX, NP = SM::NP;
  constexpr int NT = ((BX + 2) * (BY + 2) + 31) / 32 * 32;
  float *sm_f = smem;                  // [2][18][NE]
  float *sm_psi = smem + 2 * 18 * NE;  // [4][NP]

  const int tid = threadIdx.x;
  const bool active = tid < NE;
  const int lx = tid % EX, ly = tid / EX;
  const int nx = P.nx, ny = P.ny, nz = P.nz;
  const unsigned n = (unsigned)P.n, nxy = (unsigned)(nx * ny);
  const int gx = wrap(x0 + lx - 1, nx), gy = wrap(y0 + ly - 1, ny);
  const bool interior = active && lx >= 1 && lx <= BX && ly >= 1 && ly <= BY && x0 + lx - 1 < nx &&
                        y0 + ly - 1 < ny;
  const Rates<float> r(P);
  const float rho_ref = P.frho_ref, mG = -P.fG;

  // In-plane offsets (y' nx + x') of the pull sources x - e_a of this node: the
  // nine (x - ex, y - ey) combinations, computed once.  Element offsets are
  // unsigned 32-bit: 19 N < 2^32 for every box the library accepts.
  const int xm = gx == 0 ? nx - 1 : gx - 1, xp = gx == nx - 1 ? 0 : gx + 1;
  const int ym = gy == 0 ? ny - 1 : gy - 1, yp = gy == ny - 1 ? 0 : gy + 1;
  const unsigned r0 = (unsigned)(gy * nx), rm = (unsigned)(ym * nx), rp = (unsigned)(yp * nx);
  const unsigned o_00 = r0 + gx, o_m0 = r0 + xm, o_p0 = r0 + xp;  // (x-ex) with ey = 0
  const unsigned o_0m = rm + gx, o_0p = rp + gx;                 // ex = 0, y - ey = y-1 / y+1
  const unsigned o_mm = rm + xm, o_pp = rp + xp, o_mp = rp + xm, o_pm = rm + xp;

  // psi(t) tile nodes this thread copies into the ring (at most two per plane)
  constexpr int KPSI = (NP + NT - 1) / NT;
  unsigned psi_xy[KPSI];
  bool psi_ok[KPSI];
#pragma unroll
  for (int k = 0; k < KPSI; ++k) {
    const int q = tid + k * NT;
    psi_ok[k] = q < NP;
    psi_xy[k] = psi_ok[k] ? (unsigned)(wrap(x0 - 2 + q % PX, nx) + nx * wrap(y0 - 2 + q / PX, ny)) : 0u;
  }
  auto psi_slot = [&](int zp) { return sm_psi + (zp & 3) * NP; };
  auto zwrap = [&](int zp) { return zp < 0 ? zp + nz : (zp >= nz ? zp - nz : zp); };
  auto load_plane = [&](int zp, S fr[19]) {
    // pull sources of plane zp: populations with e_z = +1 come from plane zp-1, e_z = -1 from zp+1
    const unsigned zm_ = (unsigned)zwrap(zp - 1) * nxy, z0_ = (unsigned)zwrap(zp) * nxy, zp_ = (unsigned)zwrap(zp + 1) * nxy;
    fr[0] = g_in[z0_ + o_00];
    fr[1] = g_in[1u * n + z0_ + o_m0];
    fr[2] = g_in[2u * n + z0_ + o_p0];
    fr[3] = g_in[3u * n + z0_ + o_0m];
    fr[4] = g_in[4u * n + z0_ + o_0p];
    fr[5] = g_in[5u * n + zm_ + o_00];
    fr[6] = g_in[6u * n + zp_ + o_00];
    fr[7] = g_in[7u * n + z0_ + o_mm];
    fr[8] = g_in[8u * n + z0_ + o_pp];
    fr[9] = g_in[9u * n + z0_ + o_mp];
    fr[10] = g_in[10u * n + z0_ + o_pm];
    fr[11] = g_in[11u * n + zm_ + o_m0];
    fr[12] = g_in[12u * n + zp_ + o_p0];
    fr[13] = g_in[13u * n + zp_ + o_m0];
    fr[14] = g_in[14u * n + zm_ + o_p0];
    fr[15] = g_in[15u * n + zm_ + o_0m];
    fr[16] = g_in[16u * n + zp_ + o_0p];
    fr[17] = g_in[17u * n + zp_ + o_0m];
    fr[18] = g_in[18u * n + zm_ + o_0p];
  };

  // prologue: psi planes z0-2 .. z0 into the ring, populations of plane z0-1
  for (int zp = z0 - 2; zp <= z0; ++zp) {
    const unsigned zo = (unsigned)zwrap(zwrap(zp)) * nxy;  // z0 - 2 >= -2
#pragma unroll
    for (int k = 0; k < KPSI; ++k)
      if (psi_ok[k]) psi_slot(zp)[tid + k * NT] = __ldg(psi_in + zo + psi_xy[k]);
  }
  S fn[19];
  if (active) load_plane(z0 - 1, fn);
  __syncthreads();

  // partial sums of rho(t+1) - rho_ref: A for plane zz-1, B for plane zz
  float A = 0.f, B = 0.f;
  const int c = (ly + 1) * PX + (lx + 1);  // this node in the psi tile
  for (int zz = z0 - 1; zz <= z1; ++zz) {
    float *buf = sm_f + (zz & 1) * 18 * NE;
    float f[19];
#pragma unroll
    for (int a = 0; a < 19; ++a) f[a] = Storage<S>::decode(fn[a], a);
    // issue the loads of the next plane (populations, and psi plane zz+2)
    if (active && zz < z1) load_plane(zz + 1, fn);
    float pn[KPSI];
    {
      const unsigned zo = (unsigned)zwrap(zwrap(zz + 2)) * nxy;
#pragma unroll
      for (int k = 0; k < KPSI; ++k) pn[k] = psi_ok[k] ? __ldg(psi_in + zo + psi_xy[k]) : 0.f;
    }
    if (active) {
      const float *pm = psi_slot(zz - 1), *p0 = psi_slot(zz), *pp = psi_slot(zz + 1);
      float p[19];
      p[0] = p0[c];
      p[1] = p0[c + 1];        p[2] = p0[c - 1];
      p[3] = p0[c + PX];       p[4] = p0[c - PX];
      p[5] = pp[c];            p[6] = pm[c];
      p[7] = p0[c + 1 + PX];   p[8] = p0[c - 1 - PX];
      p[9] = p0[c + 1 - PX];   p[10] = p0[c - 1 + PX];
      p[11] = pp[c + 1];       p[12] = pm[c - 1];
      p[13] = pm[c + 1];       p[14] = pp[c - 1];
      p[15] = pp[c + PX];      p[16] = pm[c - PX];
      p[17] = pm[c + PX];      p[18] = pp[c - PX];
      float Sx, Sy, Sz;
      psi_gradient<float>(p, Sx, Sy, Sz);
      const float k = mG * p[0];
      const float dS4 = SIGMA ? P.fsigma_coef * (Sx * Sx + Sy * Sy + Sz * Sz) : 0.f;
      if (OP == kNonOrth || (OP == kOpRuntime && op_rt == kNonOrth))
        collide_nonorth<float>(f, rho_ref, k * Sx, k * Sy, k * Sz, dS4, r);
      else
        collide_orth<float>(f, rho_ref, k * Sx, k * Sy, k * Sz, dS4, r);
      if (interior && zz >= z0 && zz < z1) {
        const unsigned self = (unsigned)zz * nxy + o_00;
#pragma unroll
        for (int a = 0; a < 19; ++a) Storage<S>::store(g_out + (unsigned)a * n + self, a, f[a]);
      }
#pragma unroll
      for (int a = 1; a < 19; ++a) buf[(a - 1) * NE + tid] = f[a];
    }
    {
      float *dst = psi_slot(zz + 2);  // the slot of plane zz-2, no longer read
#pragma unroll
      for (int k = 0; k < KPSI; ++k)
        if (psi_ok[k]) dst[tid + k * NT] = pn[k];
    }
    __syncthreads();
    if (interior) {
      // source of direction a for this node in the extended plane: (lx - ex, ly - ey)
      const float *b = buf + tid;
      constexpr int W = -1, E = +1, Sth = -EX, N = +EX;
      // e_z = 0: a = 0 (own), 1, 2, 3, 4, 7, 8, 9, 10
      const float s_in = f[0] + (b[0 * NE + W] + b[1 * NE + E]) + (b[2 * NE + Sth] + b[3 * NE + N]) +
                         (b[6 * NE + W + Sth] + b[7 * NE + E + N]) + (b[8 * NE + W + N] + b[9 * NE + E + Sth]);
      // e_z = +1 (into plane zz+1): a = 5, 11, 14, 15, 18
      const float s_up = b[4 * NE] + (b[10 * NE + W] + b[13 * NE + E]) + (b[14 * NE + Sth] + b[17 * NE + N]);
      // e_z = -1 (into plane zz-1): a = 6, 12, 13, 16, 17
      const float s_dn = b[5 * NE] + (b[11 * NE + E] + b[12 * NE + W]) + (b[15 * NE + N] + b[16 * NE + Sth]);
      A += s_dn;  // rho(t+1) of plane zz-1 is now complete
      if (zz - 1 >= z0) {
        const double rho = P.rho_ref + (double)A;
        psi_out[(unsigned)(zz - 1) * nxy + o_00] = eos_psi<EOS, float>(rho, rho_ref + A, P, e);
      }
      A = B + s_in;
      B = s_up;
    }
  }
}

template <int PREC, int OP, bool SIGMA, int EOS, int BX, int BY>
__global__ void __launch_bounds__(((BX + 2) * (BY + 2) + 31) / 32 * 32, (one_min_blocks<BX, BY>()))
    onepass_kernel(const typename OneTypes<PREC>::S *__restrict__ g_in, typename OneTypes<PREC>::S *__restrict__ g_out,
                   const float *__restrict__ psi_in, float *__restrict__ psi_out, const KParams P, int zc,
                   unsigned *__restrict__ err) {
  extern __shared__ float smem[];
  unsigned e = 0;
  const int z0 = blockIdx.z * zc;
  onepass_tile<PREC, OP, SIGMA, EOS, BX, BY>(g_in, g_out, psi_in, psi_out, P, blockIdx.x * BX, blockIdx.y * BY, z0,
                                             min(z0 + zc, P.nz), OP, e, smem);
  if (e) atomicOr(err, e);
}

// Many boxes in one persistent launch: thread block b takes work items b,
// b + gridDim.x, ...; an item is one tile of one box and a range of planes.
template <int PREC, int EOS, int BX, int BY>
__global__ void __launch_bounds__(((BX + 2) * (BY + 2) + 31) / 32 * 32, (one_min_blocks<BX, BY>()))
    batch_onepass_kernel(const BatchBox *__restrict__ boxes, const int4 *__restrict__ items, int nitems, int parity,
                         unsigned *__restrict__ err) {
  using S = typename OneTypes<PREC>::S;
  extern __shared__ float smem[];
  __shared__ BatchBox bb;
  unsigned e = 0;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int4 w = items[it];  // (box, tx | ty << 16, z0, z1)
    __syncthreads();           // every thread is done with the previous item's descriptor
    {
      const int *src = (const int *)(boxes + w.x);
      int *dst = (int *)&bb;
      for (int k = threadIdx.x; k < (int)(sizeof(BatchBox) / sizeof(int)); k += blockDim.x) dst[k] = src[k];
    }
    __syncthreads();
    const int in = bb.cur ^ parity;
    onepass_tile<PREC, kOpRuntime, true, EOS, BX, BY>(
        (const S *)bb.g[in], (S *)bb.g[in ^ 1], bb.psi[in], bb.psi[in ^ 1], bb.P, (w.y & 0xffff) * BX,
        (w.y >> 16) * BY, w.z, w.w, bb.op, e, smem);
  }
  if (e) atomicOr(err, e);
}

template <int PREC, int OP, bool SIGMA, int EOS, int BX, int BY>
cudaError_t launch_tile(const KParams &P, const void *g_in, void *g_out, const void *psi_in, void *psi_out, int zc,
                        unsigned *err, cudaStream_t s) {
  using S = typename OneTypes<PREC>::S;
  constexpr int NT = ((BX + 2) * (BY + 2) + 31) / 32 * 32;
  constexpr size_t smem = OneSmem<BX, BY>::bytes;
  static bool attr_set = false;  // per process; the attribute is per function, not per device
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(onepass_kernel<PREC, OP, SIGMA, EOS, BX, BY>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const dim3 grid((P.nx + BX - 1) / BX, (P.ny + BY - 1) / BY, (P.nz + zc - 1) / zc);
  onepass_kernel<PREC, OP, SIGMA, EOS, BX, BY><<<grid, NT, smem, s>>>((const S *)g_in, (S *)g_out,
                                                                      (const float *)psi_in, (float *)psi_out, P, zc,
                                                                      err);
  return cudaGetLastError();
}

template <int PREC, int OP, bool SIGMA, int EOS>
cudaError_t by_tile(const KParams &P, int tile, const void *g_in, void *g_out, const void *psi_in, void *psi_out,
                    int zc, unsigned *err, cudaStream_t s) {
  switch (tile) {
    case kTile32x4: return launch_tile<PREC, OP, SIGMA, EOS, 32, 4>(P, g_in, g_out, psi_in, psi_out, zc, err, s);
    case kTile64x4: return launch_tile<PREC, OP, SIGMA, EOS, 64, 4>(P, g_in, g_out, psi_in, psi_out, zc, err, s);
    default: return launch_tile<PREC, OP, SIGMA, EOS, 32, 8>(P, g_in, g_out, psi_in, psi_out, zc, err, s);
  }
}

template <int PREC, int OP, bool SIGMA>
cudaError_t by_eos(const KParams &P, int tile, const void *g_in, void *g_out, const void *psi_in, void *psi_out, int zc,
                   unsigned *err, cudaStream_t s) {
  switch (P.eos) {
    case kEosCS: return by_tile<PREC, OP, SIGMA, kEosCS>(P, tile, g_in, g_out, psi_in, psi_out, zc, err, s);
    case kEosExp: return by_tile<PREC, OP, SIGMA, kEosExp>(P, tile, g_in, g_out, psi_in, psi_out, zc, err, s);
    default: return by_tile<PREC, OP, SIGMA, kEosNone>(P, tile, g_in, g_out, psi_in, psi_out, zc, err, s);
  }
}

template <int PREC>
cudaError_t by_op(const KParams &P, int op, bool sigma, int tile, const void *g_in, void *g_out, const void *psi_in,
                  void *psi_out, int zc, unsigned *err, cudaStream_t s) {
  if (op == kNonOrth)
    return sigma ? by_eos<PREC, kNonOrth, true>(P, tile, g_in, g_out, psi_in, psi_out, zc, err, s)
                 : by_eos<PREC, kNonOrth, false>(P, tile, g_in, g_out, psi_in, psi_out, zc, err, s);
  return sigma ? by_eos<PREC, kOrth, true>(P, tile, g_in, g_out, psi_in, psi_out, zc, err, s)
               : by_eos<PREC, kOrth, false>(P, tile, g_in, g_out, psi_in, psi_out, zc, err, s);
}

template <int PREC, int EOS, int BX, int BY>
cudaError_t batch_tile(const BatchBox *boxes, const int4 *items, int nitems, int parity, int grid, unsigned *err,
                       cudaStream_t s) {
  constexpr int NT = ((BX + 2) * (BY + 2) + 31) / 32 * 32;
  constexpr size_t smem = OneSmem<BX, BY>::bytes;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(batch_onepass_kernel<PREC, EOS, BX, BY>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  batch_onepass_kernel<PREC, EOS, BX, BY><<<grid, NT, smem, s>>>(boxes, items, nitems, parity, err);
  return cudaGetLastError();
}

template <int PREC, int EOS>
cudaError_t batch_by_tile(int tile, const BatchBox *boxes, const int4 *items, int nitems, int parity, int grid,
                          unsigned *err, cudaStream_t s) {
  switch (tile) {
    case kTile32x4: return batch_tile<PREC, EOS, 32, 4>(boxes, items, nitems, parity, grid, err, s);
    case kTile64x4: return batch_tile<PREC, EOS, 64, 4>(boxes, items, nitems, parity, grid, err, s);
    default: return batch_tile<PREC, EOS, 32, 8>(boxes, items, nitems, parity, grid, err, s);
  }
}

}  // namespace

int onepass_tile_shape(int tile, int *bx, int *by) {
  *bx = tile == kTile64x4 ? 64 : 32;
  *by = tile == kTile32x8 ? 8 : 4;
  return ((*bx + 2) * (*by + 2) + 31) / 32 * 32;
}

cudaError_t launch_batch_onepass(int precision, int eos, int tile, const BatchBox *boxes, const int4 *items,
                                 int nitems, int parity, int grid, unsigned *err, cudaStream_t s) {
  if (precision == kF32) {
    switch (eos) {
      case kEosCS: return batch_by_tile<kF32, kEosCS>(tile, boxes, items, nitems, parity, grid, err, s);
      case kEosExp: return batch_by_tile<kF32, kEosExp>(tile, boxes, items, nitems, parity, grid, err, s);
      default: return batch_by_tile<kF32, kEosNone>(tile, boxes, items, nitems, parity, grid, err, s);
    }
  }
  if (precision == kF16) {
    switch (eos) {
      case kEosCS: return batch_by_tile<kF16, kEosCS>(tile, boxes, items, nitems, parity, grid, err, s);
      case kEosExp: return batch_by_tile<kF16, kEosExp>(tile, boxes, items, nitems, parity, grid, err, s);
      default: return batch_by_tile<kF16, kEosNone>(tile, boxes, items, nitems, parity, grid, err, s);
    }
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_onepass(const KParams &P, int precision, int op, bool sigma, int tile, int zc, const void *g_in,
                           void *g_out, const void *psi_in, void *psi_out, unsigned *err, cudaStream_t s) {
  if (zc < 1) zc = 1;
  if (precision == kF32) return by_op<kF32>(P, op, sigma, tile, g_in, g_out, psi_in, psi_out, zc, err, s);
  if (precision == kF16) return by_op<kF16>(P, op, sigma, tile, g_in, g_out, psi_in, psi_out, zc, err, s);
  return cudaErrorInvalidValue;  // FP64 uses the two-pass step
}

}  // namespace lbm
