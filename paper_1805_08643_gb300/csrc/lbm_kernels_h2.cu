// Two-pass kernels for FP16 storage with two x-adjacent nodes per thread.
//
// A warp covers 64 consecutive nodes of one row.  Each thread loads the pair
// (x, x+1) of every direction with one aligned 32-bit load; the populations
// pulled from x-1 (e_x = +1) or x+2 (e_x = -1) come from the neighbouring
// lane's pair by a shuffle, and the first / last lane of the warp (or a pair
// at the periodic x boundary) loads that one value itself.  Per-node
// arithmetic is that of the one-node kernels in lbm_kernels.cu.  Needs Nx even.
#include <cuda_fp16.h>

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Row offset (y', z' part of the node index) of the pull source of direction a.
__device__ __forceinline__ int src_row(const Nbhd &nb, int a) {
  switch (a) {
    case 0: case 1: case 2: return nb.r00;
    case 3: case 7: case 10: return nb.rm0;
    case 4: case 8: case 9: return nb.rp0;
    case 5: case 11: case 14: return nb.r0m;
    case 6: case 12: case 13: return nb.r0p;
    case 15: return nb.rmm;
    case 16: return nb.rpp;
    case 17: return nb.rmp;
    default: return nb.rpm;
  }
}

__device__ __forceinline__ constexpr int ex_of(int a) {
  return (a == 1 || a == 7 || a == 9 || a == 11 || a == 13) ? 1 : (a == 2 || a == 8 || a == 10 || a == 12 || a == 14) ? -1 : 0;
}

// Pull the 19 populations of nodes xa (f0) and xa + 1 (f1), decoded to deviations.
__device__ __forceinline__ void pull_pair(const __half *__restrict__ g, unsigned n, const Nbhd &nb, int xa, int xm1,
                                          int xp2, bool valid, bool edge_prev, bool edge_next, float f0[19],
                                          float f1[19]) {
#pragma unroll
  for (int a = 0; a < 19; ++a) {
    const __half *rowp = g + (size_t)a * n + src_row(nb, a);
    const __half2 v = valid ? __ldg((const __half2 *)(rowp + xa)) : __float2half2_rn(0.f);
    const float lo = __low2float(v), hi = __high2float(v);
    float a0, a1;
    if (ex_of(a) == 0) {
      a0 = lo;
      a1 = hi;
    } else if (ex_of(a) > 0) {  // nodes pull from x - 1: (xa - 1, xa)
      float prev = __shfl_up_sync(kFull, hi, 1);
      if (edge_prev) prev = valid ? __half2float(__ldg(rowp + xm1)) : 0.f;
      a0 = prev;
      a1 = lo;
    } else {  // nodes pull from x + 1: (xa + 1, xa + 2)
      float next = __shfl_down_sync(kFull, lo, 1);
      if (edge_next) next = valid ? __half2float(__ldg(rowp + xp2)) : 0.f;
      a0 = hi;
      a1 = next;
    }
    const float w = (float)lattice_w(a);
    f0[a] = a0 * w;
    f1[a] = a1 * w;
  }
}

template <int EOS, bool DF>
__global__ void __launch_bounds__(128) psi_h2_kernel(const __half *__restrict__ g, float *__restrict__ psi,
                                                     const KParams P, unsigned *__restrict__ err) {
  const int lane = threadIdx.x;
  const int xa = 2 * (blockIdx.x * 32 + threadIdx.x), y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
  const bool valid = xa < P.nx && y < P.ny;
  const int xx = valid ? xa : 0, yy = valid ? y : 0;
  const Nbhd nb(xx, yy, z, P);
  const int xm1 = nb.xm, xp2 = xx + 2 >= P.nx ? xx + 2 - P.nx : xx + 2;
  float f0[19], f1[19];
  pull_pair(g, (unsigned)P.n, nb, xx, xm1, xp2, valid, lane == 0, lane == 31 || xx + 2 >= P.nx, f0, f1);
  if (!valid) return;
  unsigned e = 0;
  float out[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float *f = k == 0 ? f0 : f1;
    const float sax = (f[1] + f[2]) + (f[3] + f[4]) + (f[5] + f[6]);
    const float sdg = ((f[7] + f[8]) + (f[9] + f[10])) + ((f[11] + f[12]) + (f[13] + f[14])) +
                      ((f[15] + f[16]) + (f[17] + f[18]));
    const float drho = f[0] + sax + sdg;
    if (DF) {
      out[k] = eos_psi_f2<EOS>(drho, P, e);
    } else {
      out[k] = eos_psi<EOS, float>(P.rho_ref + (double)drho, P.frho_ref + drho, P, e);
    }
  }
  *(float2 *)(psi + nb.self) = make_float2(out[0], out[1]);
  if (e) atomicOr(err, e);
}

template <int OP, bool SIGMA>
__global__ void __launch_bounds__(128) fused_h2_kernel(const __half *__restrict__ g_in, __half *__restrict__ g_out,
                                                       const float *__restrict__ psi, const KParams P) {
  const int lane = threadIdx.x;
  const int xa = 2 * (blockIdx.x * 32 + threadIdx.x), y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
  const bool valid = xa < P.nx && y < P.ny;
  const int xx = valid ? xa : 0, yy = valid ? y : 0;
  const Nbhd nb0(xx, yy, z, P);
  const int xm1 = nb0.xm, xp2 = xx + 2 >= P.nx ? xx + 2 - P.nx : xx + 2;
  float f0[19], f1[19];
  pull_pair(g_in, (unsigned)P.n, nb0, xx, xm1, xp2, valid, lane == 0, lane == 31 || xx + 2 >= P.nx, f0, f1);
  if (!valid) return;
  const Nbhd nb1(xx + 1, yy, z, P);
  const Rates<float> r(P);
  const float rho_ref = P.frho_ref, mG = -P.fG;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const Nbhd &nb = k == 0 ? nb0 : nb1;
    float *f = k == 0 ? f0 : f1;
    float p[19];
#pragma unroll
    for (int a = 1; a < 19; ++a) p[a] = __ldg(psi + nb.dst(a));
    p[0] = __ldg(psi + nb.self);
    float Sx, Sy, Sz;
    psi_gradient<float>(p, Sx, Sy, Sz);
    const float kk = mG * p[0];
    const float dS4 = SIGMA ? P.fsigma_coef * (Sx * Sx + Sy * Sy + Sz * Sz) : 0.f;
    if (OP == kNonOrth)
      collide_nonorth<float>(f, rho_ref, kk * Sx, kk * Sy, kk * Sz, dS4, r);
    else
      collide_orth<float>(f, rho_ref, kk * Sx, kk * Sy, kk * Sz, dS4, r);
  }
#pragma unroll
  for (int a = 0; a < 19; ++a) {
    const float iw = lattice_inv_w(a);
    *(__half2 *)(g_out + (size_t)a * P.n + nb0.self) =
        __halves2half2(__float2half_rn(f0[a] * iw), __float2half_rn(f1[a] * iw));
  }
}

dim3 pair_grid(const KParams &P, const Launch &L) {
  return dim3((P.nx / 2 + 31) / 32, (P.ny + L.by - 1) / L.by, P.nz);
}

}  // namespace

bool h2_supported(const KParams &P) { return P.nx % 2 == 0; }

cudaError_t launch_psi_h2(const KParams &P, const void *g, void *psi, unsigned *err, const Launch &L, bool df) {
  const dim3 grid = pair_grid(P, L), block(32, L.by);
  const __half *gg = (const __half *)g;
  float *pp = (float *)psi;
  switch (P.eos) {
    case kEosCS:
      if (df) psi_h2_kernel<kEosCS, true><<<grid, block, 0, L.stream>>>(gg, pp, P, err);
      else psi_h2_kernel<kEosCS, false><<<grid, block, 0, L.stream>>>(gg, pp, P, err);
      break;
    case kEosExp:
      if (df) psi_h2_kernel<kEosExp, true><<<grid, block, 0, L.stream>>>(gg, pp, P, err);
      else psi_h2_kernel<kEosExp, false><<<grid, block, 0, L.stream>>>(gg, pp, P, err);
      break;
    default:
      psi_h2_kernel<kEosNone, false><<<grid, block, 0, L.stream>>>(gg, pp, P, err);
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_fused_h2(const KParams &P, int op, bool sigma, const void *g_in, void *g_out, const void *psi,
                            const Launch &L) {
  const dim3 grid = pair_grid(P, L), block(32, L.by);
  const __half *gi = (const __half *)g_in;
  __half *go = (__half *)g_out;
  const float *pp = (const float *)psi;
  if (op == kNonOrth) {
    if (sigma) fused_h2_kernel<kNonOrth, true><<<grid, block, 0, L.stream>>>(gi, go, pp, P);
    else fused_h2_kernel<kNonOrth, false><<<grid, block, 0, L.stream>>>(gi, go, pp, P);
  } else {
    if (sigma) fused_h2_kernel<kOrth, true><<<grid, block, 0, L.stream>>>(gi, go, pp, P);
    else fused_h2_kernel<kOrth, false><<<grid, block, 0, L.stream>>>(gi, go, pp, P);
  }
  return cudaGetLastError();
}

}  // namespace lbm
