// Two-node pieces of the D3Q15 variant (lbm_q15.cuh): populations with e_x = 0
// as one aligned pair, the others as two scalars; FP16 storage scaled by the
// D3Q15 weights; the psi stencil of Eq. 15 on D3Q15; and the per-pair fused
// and psi bodies the single-pass work list runs (as the two-pass kernels of
// lbm_kernels_pair.cu compute them, so results are equal bit for bit).
#pragma once

#include <cuda_fp16.h>

#include "lbm_device.cuh"
#include "lbm_pair.cuh"
#include "lbm_q15.cuh"

namespace lbm {

template <typename S> struct PairIO15 {
  static __device__ __forceinline__ V2 decode(float2 v, int a) { return PairIO<S>::decode(v, a); }
  static __device__ __forceinline__ void st2(S *p, int a, V2 v) { PairIO<S>::st2(p, a, v); }
};
template <> struct PairIO15<__half> {
  static __device__ __forceinline__ V2 decode(float2 v, int a) { return V2(v) * V2(q15::w(a)); }
  static __device__ __forceinline__ void st2(__half *p, int a, V2 v) {
    *(__half2 *)p = __float22half2_rn(V2(v * V2((double)q15::inv_w(a))).v);
  }
};

// Row offset (y', z' part) of the pull source of direction a (x - e_a).
__device__ __forceinline__ int src_row15(const Nbhd &nb, int a) {
  switch (a) {
    case 0: case 1: case 2: return nb.r00;
    case 3: return nb.rm0;
    case 4: return nb.rp0;
    case 5: return nb.r0m;
    case 6: return nb.r0p;
    case 7: case 13: return nb.rmm;
    case 8: case 14: return nb.rpp;
    case 9: case 12: return nb.rmp;
    default: return nb.rpm;
  }
}

// Pull of both nodes' 15 populations; Ld: PairIO<S> (read-only path) or
// L2Load<S> (populations written earlier in the same launch).
template <typename S, typename Ld = PairIO<S>>
__device__ __forceinline__ void pull_pair15(const S *__restrict__ g, unsigned n, const Nbhd &nb, const PairX &px,
                                            V2 f[q15::kQ]) {
#pragma unroll
  for (int a = 0; a < q15::kQ; ++a) {
    const S *rowp = g + (size_t)a * n + src_row15(nb, a);
    float2 v;
    if (q15::ex(a) == 0)
      v = Ld::ld2(rowp + px.x);
    else if (q15::ex(a) > 0)
      v = make_float2(Ld::ld1(rowp + px.xm1), Ld::ld1(rowp + px.x));
    else
      v = make_float2(Ld::ld1(rowp + px.x + 1), Ld::ld1(rowp + px.xp2));
    f[a] = PairIO15<S>::decode(v, a);
  }
}

// psi(x + e_a) of both nodes, p[a] (Eq. 15 stencil on D3Q15).
__device__ __forceinline__ void gather_psi_pair15(const float *__restrict__ psi, const Nbhd &nb, const PairX &px,
                                                  V2 p[q15::kQ]) {
  // centre pair, and the pairs shifted by +1 and -1 in x
  auto row3 = [&](int row, V2 &c, V2 &plus, V2 &minus) {
    const float2 m = __ldg((const float2 *)(psi + row + px.x));
    const float l = __ldg(psi + row + px.xm1), r = __ldg(psi + row + px.xp2);
    c = V2(m);
    plus = V2(m.y, r);
    minus = V2(l, m.x);
  };
  auto row1 = [&](int row) { return V2(__ldg((const float2 *)(psi + row + px.x))); };
  V2 unused;
  row3(nb.r00, p[0], p[1], p[2]);
  p[3] = row1(nb.rp0);
  p[4] = row1(nb.rm0);
  p[5] = row1(nb.r0p);
  p[6] = row1(nb.r0m);
  row3(nb.rpp, unused, p[7], p[13]);
  row3(nb.rmm, unused, p[14], p[8]);
  row3(nb.rpm, unused, p[9], p[12]);
  row3(nb.rmp, unused, p[11], p[10]);
}

// Fused pass of one pair on D3Q15 (pull, force from the psi stencil, collision, store).
template <typename S, bool SIGMA>
__device__ __forceinline__ void fused_pair15_at(const S *__restrict__ g_in, S *__restrict__ g_out,
                                                const float *__restrict__ psi, const KParams &P, int x, int y, int z) {
  const PairX px = pair_x(P, x);
  const Nbhd nb(x, y, z, P);
  V2 f[q15::kQ];
  pull_pair15<S>(g_in, (unsigned)P.n, nb, px, f);
  V2 Fx, Fy, Fz, dS4;
  {
    V2 p[q15::kQ];
    gather_psi_pair15(psi, nb, px, p);
    V2 Sx, Sy, Sz;
    q15::psi_gradient<V2>(p, Sx, Sy, Sz);
    const V2 kk = V2((double)-P.fG) * p[0];
    dS4 = SIGMA ? V2(V2((double)P.fsigma_coef) * V2(Sx * Sx + Sy * Sy + Sz * Sz)) : V2(0.0);
    Fx = kk * Sx;
    Fy = kk * Sy;
    Fz = kk * Sz;
  }
  q15::collide<V2>(f, V2((double)P.frho_ref), Fx, Fy, Fz, dS4, Rates<V2>(P));
#pragma unroll
  for (int a = 0; a < q15::kQ; ++a) PairIO15<S>::st2(g_out + (size_t)a * P.n + nb.self, a, f[a]);
}

// psi of one pair on D3Q15 from populations written earlier in the same launch (pulls through L2).
template <typename S, int EOS, bool DF, bool ICVT = true>
__device__ __forceinline__ void psi_pair15_at_l2(const S *__restrict__ g, float *__restrict__ psi, const KParams &P,
                                                 int x, int y, int z, unsigned &e) {
  const PairX px = pair_x(P, x);
  const Nbhd nb(x, y, z, P);
  V2 f[q15::kQ];
  pull_pair15<S, L2Load<S>>(g, (unsigned)P.n, nb, px, f);
  *(float2 *)(psi + nb.self) = psi_pair<EOS, DF, ICVT>(q15::drho(f), P, e);
}

}  // namespace lbm
