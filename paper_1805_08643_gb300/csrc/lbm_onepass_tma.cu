// Single-pass step with bulk asynchronous copies (FP32 storage).
//
// Same algorithm as lbm_onepass.cu (x-y tile marched along z, collisions
// recomputed on a one-node ring, rho(t+1) gathered through shared memory,
// psi(t+1) written by the kernel), but the data movement runs on the copy
// engine instead of per-thread loads and stores:
//  * For every plane, the rows of a window x in [x0-4, x0+BX+4), y in
//    [y0-2, y0+BY+2) of each of the 19 population arrays (at the plane each
//    direction streams from) and of psi(t) are brought into shared memory by
//    cp.async.bulk row copies that complete on an mbarrier.  A row that crosses
//    the periodic x boundary is split into aligned pieces.  Copies run two
//    planes ahead of the collisions (two stages).
//  * The post-collision populations of the interior rows leave shared memory
//    through cp.async.bulk shared->global copies.
// Every wait is bounded: a wait that gives up sets kErrTimeout and the thread
// goes on, so no thread can hang at a barrier.
// Requirements (checked by the launcher): nx % 4 == 0 and nx >= BX + 8.
#include <cuda_runtime.h>

#include "lbm_async.cuh"
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {
namespace {

__device__ __forceinline__ int wrapi(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

template <int BX, int BY> struct TmaSmem {
  static constexpr int EX = BX + 2, EY = BY + 2;  // extended tile (threads)
  static constexpr int WX = BX + 8, WY = BY + 4;  // copy window (x aligned to 4 elements)
  static constexpr int WIN = WX * WY;             // one array's window, elements
  static constexpr int STAGE = 20 * WIN;          // 19 populations + psi
  static constexpr int FX = BX + 8;               // pitch of the f* exchange rows
  static constexpr int FSTAR = 19 * EY * FX;      // one f* buffer
  static constexpr size_t bytes = sizeof(float) * (2 * STAGE + 2 * FSTAR + 4 * WIN) + 64;
};

// Direction components (Eq. 2).
__device__ __forceinline__ constexpr int EXd(int a) {
  return (a == 1 || a == 7 || a == 9 || a == 11 || a == 13) ? 1 : (a == 2 || a == 8 || a == 10 || a == 12 || a == 14) ? -1 : 0;
}
__device__ __forceinline__ constexpr int EYd(int a) {
  return (a == 3 || a == 7 || a == 10 || a == 15 || a == 17) ? 1 : (a == 4 || a == 8 || a == 9 || a == 16 || a == 18) ? -1 : 0;
}
__device__ __forceinline__ constexpr int EZd(int a) {
  return (a == 5 || a == 11 || a == 14 || a == 15 || a == 18) ? 1 : (a == 6 || a == 12 || a == 13 || a == 16 || a == 17) ? -1 : 0;
}

template <int OP, bool SIGMA, int EOS, int BX, int BY>
__global__ void __launch_bounds__(((BX + 2) * (BY + 2) + 31) / 32 * 32, 1)
    onepass_tma_kernel(const float *__restrict__ g_in, float *__restrict__ g_out, const float *__restrict__ psi_in,
                       float *__restrict__ psi_out, const KParams P, int zc, unsigned *__restrict__ err) {
  using SM = TmaSmem<BX, BY>;
  constexpr int EX = SM::EX, EY = SM::EY, WX = SM::WX, WY = SM::WY, WIN = SM::WIN, FX = SM::FX;
  extern __shared__ __align__(128) float smem[];
  float *stage = smem;                       // [2][20][WY][WX]
  float *fstar = stage + 2 * SM::STAGE;      // [2][19][EY][FX]
  float *ring = fstar + 2 * SM::FSTAR;       // [4][WY][WX]  psi(t) planes
  unsigned long long *bar = (unsigned long long *)(ring + 4 * WIN);  // [2]

  const int tid = threadIdx.x;
  const bool active = tid < EX * EY;
  const int lx = tid % EX, ly = tid / EX;
  const int nx = P.nx, ny = P.ny, nz = P.nz;
  const unsigned n = (unsigned)P.n, nxy = (unsigned)(nx * ny);
  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
  const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, nz);
  const int gx = wrapi(x0 + lx - 1, nx), gy = wrapi(y0 + ly - 1, ny);
  const bool interior = active && lx >= 1 && lx <= BX && ly >= 1 && ly <= BY && x0 + lx - 1 < nx && y0 + ly - 1 < ny;
  const Rates<float> r(P);
  const float rho_ref = P.frho_ref, mG = -P.fG;
  unsigned e = 0;

  // One copy job per thread: window row `row` of array `arr` (0..18 populations, 19 psi).
  const int job = tid;
  const bool copier = job < 20 * WY;
  const int arr = job / WY, row = job % WY;
  const int ysrc = wrapi(y0 - 2 + row, ny);
  // x pieces of a window row: [xs, xs + len) of the domain -> window column col
  int px[3], pl[3], pc[3], npieces = 0;
  {
    int xs = x0 - 4, col = 0, left = WX;
    while (left > 0) {
      const int xw = wrapi(xs, nx);
      const int len = min(left, nx - xw);
      px[npieces] = xw;
      pl[npieces] = len;
      pc[npieces] = col;
      ++npieces;
      xs += len;
      col += len;
      left -= len;
    }
  }
  const unsigned stage_bytes_pop = 19u * WIN * sizeof(float), psi_bytes = (unsigned)(WIN * sizeof(float));

  // issue the copies of plane zp into stage s: populations (if pop), psi plane zq into the ring (if psi)
  auto issue = [&](int s, int zp, bool pop, int zq, bool psi) {
    if (!copier) return;
    float *dst;
    const float *src;
    if (arr < 19) {
      if (!pop) return;
      const int a = arr;
      const int ez = a == 0 ? 0 : (EZd(a));
      const unsigned zs = (unsigned)wrapi(zp - ez, nz);
      dst = stage + s * SM::STAGE + a * WIN + row * WX;
      src = g_in + (size_t)a * n + zs * nxy + (unsigned)ysrc * nx;
    } else {
      if (!psi) return;
      dst = ring + (zq & 3) * WIN + row * WX;
      src = psi_in + (unsigned)wrapi(zq, nz) * nxy + (unsigned)ysrc * nx;
    }
    for (int k = 0; k < npieces; ++k)
      bulk_g2s(dst + pc[k], src + px[k], (unsigned)pl[k] * sizeof(float), &bar[s]);
  };

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_async_smem();
  }
  __syncthreads();
  // prologue: stage of plane z0-1 with psi planes z0-2..z0; stage of plane z0 with psi plane z0+1
  const int s0 = (z0 - 1) & 1, s1 = z0 & 1;
  if (tid == 0) {
    mbar_arrive_expect_tx(&bar[s0], stage_bytes_pop + 3 * psi_bytes);
    mbar_arrive_expect_tx(&bar[s1], stage_bytes_pop + psi_bytes);
  }
  __syncthreads();
  issue(s0, z0 - 1, true, z0 - 2, true);
  if (copier && arr == 19) {
    issue(s0, z0 - 1, false, z0 - 1, true);
    issue(s0, z0 - 1, false, z0, true);
  }
  issue(s1, z0, true, z0 + 1, true);
  unsigned phase[2] = {0u, 0u};

  float A = 0.f, B = 0.f;  // partial rho(t+1) - rho_ref of planes zz-1 and zz
  bool stored_last = false;
  for (int zz = z0 - 1; zz <= z1; ++zz) {
    const int s = zz & 1;
    if (!mbar_wait(&bar[s], phase[s], P.spin_limit)) e |= kErrTimeout;
    phase[s] ^= 1u;
    float f[19];
    float *fs = fstar + s * SM::FSTAR;
    if (active) {
      const float *st = stage + s * SM::STAGE;
      const int base = (ly + 1) * WX + (lx + 3);  // window cell of this node
#pragma unroll
      for (int a = 0; a < 19; ++a) f[a] = st[a * WIN + base - EYd(a) * WX - EXd(a)];
      const float *pm = ring + ((zz - 1) & 3) * WIN + base, *p0 = ring + (zz & 3) * WIN + base,
                  *pp = ring + ((zz + 1) & 3) * WIN + base;
      float p[19];
      p[0] = p0[0];
#pragma unroll
      for (int a = 1; a < 19; ++a) {
        const float *pl_ = EZd(a) > 0 ? pp : (EZd(a) < 0 ? pm : p0);
        p[a] = pl_[EYd(a) * WX + EXd(a)];
      }
      float Sx, Sy, Sz;
      psi_gradient<float>(p, Sx, Sy, Sz);
      const float k = mG * p[0];
      const float dS4 = SIGMA ? P.fsigma_coef * (Sx * Sx + Sy * Sy + Sz * Sz) : 0.f;
      if (OP == kNonOrth)
        collide_nonorth<float>(f, rho_ref, k * Sx, k * Sy, k * Sz, dS4, r);
      else
        collide_orth<float>(f, rho_ref, k * Sx, k * Sy, k * Sz, dS4, r);
#pragma unroll
      for (int a = 0; a < 19; ++a) fs[(a * EY + ly) * FX + lx + 3] = f[a];
    }
    // the bulk stores issued in the previous plane must have read their rows
    if (stored_last) bulk_wait_read();
    fence_async_smem();
    // arm this stage for the plane two ahead before anyone issues its copies
    const bool next_pop = zz + 2 <= z1, next_psi = zz + 3 <= z1 + 1;
    if (tid == 0 && next_pop)
      mbar_arrive_expect_tx(&bar[s], stage_bytes_pop + (next_psi ? psi_bytes : 0u));
    __syncthreads();
    if (next_pop) issue(s, zz + 2, true, zz + 3, next_psi);
    // interior rows of f* go out (planes z0 .. z1-1 only)
    stored_last = false;
    if (zz >= z0 && zz < z1 && tid < 19 * BY) {
      const int a = tid / BY, yy = tid % BY;
      if (y0 + yy < ny) {
        const int w = min(BX, nx - x0);
        float *dst = g_out + (size_t)a * n + (unsigned)zz * nxy + (unsigned)(y0 + yy) * nx + x0;
        bulk_s2g(dst, fs + (a * EY + yy + 1) * FX + 4, (unsigned)w * sizeof(float));
        bulk_commit();
        stored_last = true;
      }
    }
    if (interior) {
      const float *b = fs + ly * FX + lx + 3;
      constexpr int DY = FX, PL = EY * FX;  // row and direction strides in the exchange buffer
      auto at = [&](int a, int dx, int dy) { return b[a * PL + dy * DY + dx]; };
      // source of direction a for this node: (lx - ex, ly - ey)
      const float s_in = f[0] + (at(1, -1, 0) + at(2, 1, 0)) + (at(3, 0, -1) + at(4, 0, 1)) +
                         (at(7, -1, -1) + at(8, 1, 1)) + (at(9, -1, 1) + at(10, 1, -1));
      const float s_up = at(5, 0, 0) + (at(11, -1, 0) + at(14, 1, 0)) + (at(15, 0, -1) + at(18, 0, 1));
      const float s_dn = at(6, 0, 0) + (at(12, 1, 0) + at(13, -1, 0)) + (at(16, 0, 1) + at(17, 0, -1));
      A += s_dn;
      if (zz - 1 >= z0) {
        const double rho = P.rho_ref + (double)A;
        psi_out[(unsigned)(zz - 1) * nxy + (unsigned)gy * nx + gx] = eos_psi<EOS, float>(rho, rho_ref + A, P, e);
      }
      A = B + s_in;
      B = s_up;
    }
  }
  bulk_wait_all();
  if (e) atomicOr(err, e);
}

template <int OP, bool SIGMA, int EOS>
cudaError_t launch_t(const KParams &P, const void *g_in, void *g_out, const void *psi_in, void *psi_out, int zc,
                     unsigned *err, cudaStream_t s) {
  constexpr int BX = 32, BY = 8;
  constexpr int NT = ((BX + 2) * (BY + 2) + 31) / 32 * 32;
  constexpr size_t smem = TmaSmem<BX, BY>::bytes;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(onepass_tma_kernel<OP, SIGMA, EOS, BX, BY>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const dim3 grid((P.nx + BX - 1) / BX, (P.ny + BY - 1) / BY, (P.nz + zc - 1) / zc);
  onepass_tma_kernel<OP, SIGMA, EOS, BX, BY><<<grid, NT, smem, s>>>((const float *)g_in, (float *)g_out,
                                                                    (const float *)psi_in, (float *)psi_out, P, zc,
                                                                    err);
  return cudaGetLastError();
}

template <int OP, bool SIGMA>
cudaError_t by_eos_t(const KParams &P, const void *g_in, void *g_out, const void *psi_in, void *psi_out, int zc,
                     unsigned *err, cudaStream_t s) {
  switch (P.eos) {
    case kEosCS: return launch_t<OP, SIGMA, kEosCS>(P, g_in, g_out, psi_in, psi_out, zc, err, s);
    case kEosExp: return launch_t<OP, SIGMA, kEosExp>(P, g_in, g_out, psi_in, psi_out, zc, err, s);
    default: return launch_t<OP, SIGMA, kEosNone>(P, g_in, g_out, psi_in, psi_out, zc, err, s);
  }
}

}  // namespace

bool onepass_tma_supported(const KParams &P, int precision) {
  return precision == kF32 && P.nx % 4 == 0 && P.nx >= 32 + 8;
}

cudaError_t launch_onepass_tma(const KParams &P, int precision, int op, bool sigma, int zc, const void *g_in,
                               void *g_out, const void *psi_in, void *psi_out, unsigned *err, cudaStream_t s) {
  if (!onepass_tma_supported(P, precision)) return cudaErrorInvalidValue;
  if (zc < 1) zc = 1;
  if (op == kNonOrth)
    return sigma ? by_eos_t<kNonOrth, true>(P, g_in, g_out, psi_in, psi_out, zc, err, s)
                 : by_eos_t<kNonOrth, false>(P, g_in, g_out, psi_in, psi_out, zc, err, s);
  return sigma ? by_eos_t<kOrth, true>(P, g_in, g_out, psi_in, psi_out, zc, err, s)
               : by_eos_t<kOrth, false>(P, g_in, g_out, psi_in, psi_out, zc, err, s);
}

}  // namespace lbm
