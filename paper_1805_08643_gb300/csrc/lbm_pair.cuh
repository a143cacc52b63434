// Pair access for the kernels that give each thread two x-adjacent nodes
// (x even, Nx even): loads and stores of stored populations as pairs, the pull
// of both nodes' 19 populations (Eq. 5), their density, psi, force and
// collision on packed FP32 pairs (V2).
#pragma once

#include <cuda_fp16.h>

#include "lbm_device.cuh"

namespace lbm {

// Loads and stores of a pair of stored populations, decoded to FP32 deviations.
template <typename S> struct PairIO;
template <> struct PairIO<float> {
  static __device__ __forceinline__ float2 ld2(const float *p) { return __ldg((const float2 *)p); }
  static __device__ __forceinline__ float ld1(const float *p) { return __ldg(p); }
  static __device__ __forceinline__ V2 decode(float2 v, int a) { (void)a; return V2(v); }
  static __device__ __forceinline__ void st2(float *p, int a, V2 v) { (void)a; *(float2 *)p = v.v; }
};
template <> struct PairIO<__half> {
  static __device__ __forceinline__ float2 ld2(const __half *p) { return __half22float2(__ldg((const __half2 *)p)); }
  static __device__ __forceinline__ float ld1(const __half *p) { return __half2float(__ldg(p)); }
  static __device__ __forceinline__ V2 decode(float2 v, int a) { return V2(v) * V2(lattice_w(a)); }
  static __device__ __forceinline__ void st2(__half *p, int a, V2 v) {
    *(__half2 *)p = __float22half2_rn(V2(v * V2((double)lattice_inv_w(a))).v);
  }
};

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

// x positions of a pair: x (even), x - 1 and x + 2 wrapped periodically.
struct PairX {
  int x, xm1, xp2;
};

// Pull the 19 deviations of nodes x and x + 1 (Eq. 5).  Populations with
// e_x = 0 come from an aligned pair of the source row, those with e_x = +1
// from (x-1, x) and those with e_x = -1 from (x+1, x+2), read as two scalars.
template <typename S>
__device__ __forceinline__ void pull_pair(const S *__restrict__ g, unsigned n, const Nbhd &nb, const PairX &px,
                                          V2 f[19]) {
#pragma unroll
  for (int a = 0; a < 19; ++a) {
    const S *rowp = g + (size_t)a * n + src_row(nb, a);
    float2 v;
    if (ex_of(a) == 0)
      v = PairIO<S>::ld2(rowp + px.x);
    else if (ex_of(a) > 0)
      v = make_float2(PairIO<S>::ld1(rowp + px.xm1), PairIO<S>::ld1(rowp + px.x));
    else
      v = make_float2(PairIO<S>::ld1(rowp + px.x + 1), PairIO<S>::ld1(rowp + px.xp2));
    f[a] = PairIO<S>::decode(v, a);
  }
}

// rho - rho_ref of both nodes: the sum of the pulled deviations (Eq. 6).
__device__ __forceinline__ V2 drho_pair(const V2 f[19]) {
  const V2 sax = (f[1] + f[2]) + (f[3] + f[4]) + (f[5] + f[6]);
  const V2 sdg = ((f[7] + f[8]) + (f[9] + f[10])) + ((f[11] + f[12]) + (f[13] + f[14])) +
                 ((f[15] + f[16]) + (f[17] + f[18]));
  return f[0] + sax + sdg;
}

// psi of both nodes from rho - rho_ref; DF selects the compensated-FP32 radicand.
template <int EOS, bool DF, bool ICVT = true>
__device__ __forceinline__ float2 psi_pair(V2 drho, const KParams &P, unsigned &e) {
  float out[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float d = k == 0 ? drho.v.x : drho.v.y;
    if (DF)
      out[k] = eos_psi_f2<EOS>(d, P, e);
    else
      out[k] = eos_psi_d<EOS, ICVT>(d, P, e);
  }
  return make_float2(out[0], out[1]);
}

// Force of both nodes (Eq. 15) and the Eq. 16 term (when SIGMA) from
// p[a] = psi(x + e_a).
template <bool SIGMA>
__device__ __forceinline__ void force_pair(const V2 p[19], const KParams &P, V2 &Fx, V2 &Fy, V2 &Fz, V2 &dS4) {
  V2 Sx, Sy, Sz;
  psi_gradient<V2>(p, Sx, Sy, Sz);
  const V2 kk = V2((double)-P.fG) * p[0];
  dS4 = SIGMA ? V2(V2((double)P.fsigma_coef) * V2(Sx * Sx + Sy * Sy + Sz * Sz)) : V2(0.0);
  Fx = kk * Sx;
  Fy = kk * Sy;
  Fz = kk * Sz;
}

// Collision of both nodes with a given force.  OP is kOrth, kNonOrth or 2 (then op_rt picks).
template <int OP>
__device__ __forceinline__ void collide_pair(V2 f[19], V2 Fx, V2 Fy, V2 Fz, V2 dS4, const KParams &P,
                                             const Rates<V2> &r, int op_rt) {
  if (OP == kNonOrth || (OP == 2 && op_rt == kNonOrth))
    collide_nonorth<V2>(f, V2((double)P.frho_ref), Fx, Fy, Fz, dS4, r);
  else
    collide_orth<V2>(f, V2((double)P.frho_ref), Fx, Fy, Fz, dS4, r);
}

// Both of the above.
template <int OP, bool SIGMA>
__device__ __forceinline__ void force_collide_pair(V2 f[19], const V2 p[19], const KParams &P, const Rates<V2> &r,
                                                   int op_rt) {
  V2 Fx, Fy, Fz, dS4;
  force_pair<SIGMA>(p, P, Fx, Fy, Fz, dS4);
  collide_pair<OP>(f, Fx, Fy, Fz, dS4, P, r, op_rt);
}

// Loads through L2 only, for populations written by other blocks earlier in
// the same launch (the non-coherent read-only path could hold stale lines).
template <typename S> struct L2Load;
template <> struct L2Load<float> {
  static __device__ __forceinline__ float2 ld2(const float *p) { return __ldcg((const float2 *)p); }
  static __device__ __forceinline__ float ld1(const float *p) { return __ldcg(p); }
};
template <> struct L2Load<__half> {
  static __device__ __forceinline__ float2 ld2(const __half *p) { return __half22float2(__ldcg((const __half2 *)p)); }
  static __device__ __forceinline__ float ld1(const __half *p) { return __half2float(__ldcg(p)); }
};

// The pair (x, x+1), x even, of row y in plane z with its periodic x neighbours.
__device__ __forceinline__ PairX pair_x(const KParams &P, int x) {
  return PairX{x, x == 0 ? P.nx - 1 : x - 1, x + 2 >= P.nx ? x + 2 - P.nx : x + 2};
}

// Fused pass of one pair as the two-pass fused kernel computes it (Eqs. 4-6,
// 15, pull streaming of Eq. 5), with the force taken from psi before the
// populations are pulled: the two sets of 19 pairs are never live together,
// which keeps the registers of the single-pass kernels down.  The arithmetic
// and its order are those of fused_pair_kernel, so the results are equal bit
// for bit.
template <typename S, int OP, bool SIGMA, bool FORCE_FIRST = true>
__device__ __forceinline__ void fused_pair_at(const S *__restrict__ g_in, S *__restrict__ g_out,
                                              const float *__restrict__ psi, const KParams &P, int x, int y, int z,
                                              const Rates<V2> &r) {
  const PairX px = pair_x(P, x);
  const Nbhd nb(x, y, z, P);
  V2 f[19];
  // without FORCE_FIRST both sets of loads are issued before either is used
  // (one memory round trip, more registers)
  if (!FORCE_FIRST) pull_pair<S>(g_in, (unsigned)P.n, nb, px, f);
  V2 Fx, Fy, Fz, dS4;
  {
    V2 p[19];
    auto row3 = [&](int row, V2 &c, V2 &plus, V2 &minus) {
      const float2 m = __ldg((const float2 *)(psi + row + px.x));
      const float l = __ldg(psi + row + px.xm1), rr = __ldg(psi + row + px.xp2);
      c = V2(m);
      plus = V2(m.y, rr);
      minus = V2(l, m.x);
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
    force_pair<SIGMA>(p, P, Fx, Fy, Fz, dS4);
  }
  if (FORCE_FIRST) pull_pair<S>(g_in, (unsigned)P.n, nb, px, f);
  collide_pair<OP>(f, Fx, Fy, Fz, dS4, P, r, OP);
#pragma unroll
  for (int a = 0; a < 19; ++a) PairIO<S>::st2(g_out + (size_t)a * P.n + nb.self, a, f[a]);
}

// psi of one pair from populations written earlier in the same launch (the
// psi pass of psi_pair_kernel, pulls through L2).
template <typename S, int EOS, bool DF, bool ICVT = true>
__device__ __forceinline__ void psi_pair_at_l2(const S *__restrict__ g, float *__restrict__ psi, const KParams &P,
                                               int x, int y, int z, unsigned &e) {
  const PairX px = pair_x(P, x);
  const Nbhd nb(x, y, z, P);
  V2 f[19];
#pragma unroll
  for (int a = 0; a < 19; ++a) {
    const S *rowp = g + (size_t)a * P.n + src_row(nb, a);
    float2 v;
    if (ex_of(a) == 0)
      v = L2Load<S>::ld2(rowp + px.x);
    else if (ex_of(a) > 0)
      v = make_float2(L2Load<S>::ld1(rowp + px.xm1), L2Load<S>::ld1(rowp + px.x));
    else
      v = make_float2(L2Load<S>::ld1(rowp + px.x + 1), L2Load<S>::ld1(rowp + px.xp2));
    f[a] = PairIO<S>::decode(v, a);
  }
  *(float2 *)(psi + nb.self) = psi_pair<EOS, DF, ICVT>(drho_pair(f), P, e);
}

// Cross-block signalling inside one launch: a release increment of a
// completion counter (after a block barrier, by one thread: the barrier and the
// fence make every thread's earlier stores visible first) and an acquire load.
__device__ __forceinline__ void counter_release_add(int *c, int v) {
  asm volatile("fence.acq_rel.gpu;\n\tred.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(c), "r"(v) : "memory");
}
__device__ __forceinline__ int counter_acquire(const int *c) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(c) : "memory");
  return v;
}

}  // namespace lbm
