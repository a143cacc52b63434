// D3Q15 variant of the non-orthogonal operator.  The paper builds its
// operator on D3Q19 and states that a D3Q15 one follows the same construction
// (Sec. II A); this is that construction:
//
//   velocities   rest; +-x, +-y, +-z (Eq. 2 order); corners
//                (+,+,+) (-,-,-) (+,+,-) (-,-,+) (+,-,+) (-,+,-) (-,+,+) (+,-,-)
//   basis        the raw monomials of Eqs. 7-10 on these velocities: 1, e_x,
//                e_y, e_z | |e|^2, 3e_x^2 - |e|^2, e_y^2 - e_z^2, e_x e_y,
//                e_x e_z, e_y e_z | e_x^2 e_y, e_x e_y^2, e_x^2 e_z, e_x e_y e_z
//                | e_x^2 e_y^2.  (On D3Q15 e_x^2 e_y = e_y e_z^2 and its two
//                analogues coincide, the three Eq. 10 vectors are one, and
//                e_x e_y e_z, zero on D3Q19, joins the basis.)
//   equilibria   Eq. 13 values of the D3Q19 rows each vector equals (their
//   and forcing  mean where several coincide: phi + (2/3) rho c_s^2 |u|^2 and
//                (4/3) c_s^2 F.u for e_x^2 e_y^2); zero for e_x e_y e_z
//   rates        1 (conserved), s_e, s_nu x5, s_q x4, s_pi  (Eq. 11 analogue)
//   force        Eq. 15 with weights 1/3 (axes), 1/24 (corners)
//
// The eight corner moments (count, e_x e_y, e_x e_z, e_y e_z, the corner parts
// of e_x, e_y, e_z, and e_x e_y e_z) are a 3-D Walsh-Hadamard transform of the
// corner populations, evaluated with three butterfly stages in each direction;
// the axis populations meet only |e|^2, the two normal-stress rows, the
// third-order rows and the corner count.
#pragma once

#include <cuda_fp16.h>

#include "lbm_device.cuh"

namespace lbm {
namespace q15 {

constexpr int kQ = 15;

// rest-state weights: f_a = w_a rho = M^-1 m_eq(rho, 0)
__device__ __forceinline__ constexpr double w(int a) { return a == 0 ? 2.0 / 9.0 : (a < 7 ? 1.0 / 9.0 : 1.0 / 72.0); }
__device__ __forceinline__ constexpr float inv_w(int a) { return a == 0 ? 4.5f : (a < 7 ? 9.0f : 72.0f); }

__device__ __forceinline__ constexpr int ex(int a) {
  return (a == 1 || a == 7 || a == 9 || a == 11 || a == 14) ? 1 : (a == 2 || a == 8 || a == 10 || a == 12 || a == 13) ? -1 : 0;
}
__device__ __forceinline__ constexpr int ey(int a) {
  return (a == 3 || a == 7 || a == 9 || a == 12 || a == 13) ? 1 : (a == 4 || a == 8 || a == 10 || a == 11 || a == 14) ? -1 : 0;
}
__device__ __forceinline__ constexpr int ez(int a) {
  return (a == 5 || a == 7 || a == 10 || a == 11 || a == 13) ? 1 : (a == 6 || a == 8 || a == 9 || a == 12 || a == 14) ? -1 : 0;
}

// Node x - e_a: where population a of node x is pulled from (Eq. 5).
__device__ __forceinline__ int src(const Nbhd &nb, int a) {
  switch (a) {
    case 0: return nb.r00 + nb.x;
    case 1: return nb.r00 + nb.xm;   case 2: return nb.r00 + nb.xp;
    case 3: return nb.rm0 + nb.x;    case 4: return nb.rp0 + nb.x;
    case 5: return nb.r0m + nb.x;    case 6: return nb.r0p + nb.x;
    case 7: return nb.rmm + nb.xm;   case 8: return nb.rpp + nb.xp;
    case 9: return nb.rmp + nb.xm;   case 10: return nb.rpm + nb.xp;
    case 11: return nb.rpm + nb.xm;  case 12: return nb.rmp + nb.xp;
    case 13: return nb.rmm + nb.xp;  default: return nb.rpp + nb.xm;
  }
}

// Node x + e_a: the neighbour read by the interaction force (Eq. 15).
__device__ __forceinline__ int dst(const Nbhd &nb, int a) {
  switch (a) {
    case 0: return nb.r00 + nb.x;
    case 1: return nb.r00 + nb.xp;   case 2: return nb.r00 + nb.xm;
    case 3: return nb.rp0 + nb.x;    case 4: return nb.rm0 + nb.x;
    case 5: return nb.r0p + nb.x;    case 6: return nb.r0m + nb.x;
    case 7: return nb.rpp + nb.xp;   case 8: return nb.rmm + nb.xm;
    case 9: return nb.rpm + nb.xp;   case 10: return nb.rmp + nb.xm;
    case 11: return nb.rmp + nb.xp;  case 12: return nb.rpm + nb.xm;
    case 13: return nb.rpp + nb.xm;  default: return nb.rmm + nb.xp;
  }
}

// Stored populations: the deviation f_a - w_a rho_ref (FP16: divided by w_a).
template <typename S> struct Storage {
  static __device__ __forceinline__ typename lbm::Storage<S>::Compute load(const S *p, int a) {
    return lbm::Storage<S>::load(p, a);
  }
  template <typename T> static __device__ __forceinline__ void store(S *p, int a, T v) { lbm::Storage<S>::store(p, a, v); }
};
template <> struct Storage<__half> {
  static __device__ __forceinline__ float load(const __half *p, int a) { return __half2float(__ldg(p)) * (float)w(a); }
  template <typename T> static __device__ __forceinline__ void store(__half *p, int a, T v) {
    *p = __float2half_rn((float)v * inv_w(a));
  }
};

// rho - rho_ref: the sum of the deviations, in the order of the forward chain.
template <typename T>
__device__ __forceinline__ T drho(const T f[kQ]) {
  const T sax = (f[1] + f[2]) + (f[3] + f[4]) + (f[5] + f[6]);
  const T cor = ((f[7] + f[8]) + (f[9] + f[10])) + ((f[11] + f[12]) + (f[13] + f[14]));
  return f[0] + sax + cor;
}

// S = sum_a w_a psi(x + e_a) e_a with w = 1/3 (axes), 1/24 (corners);
// F = -G psi(x) S (Eq. 15).  p[a] = psi(x + e_a).
template <typename T>
__device__ __forceinline__ void psi_gradient(const T p[kQ], T &Sx, T &Sy, T &Sz) {
  const T d78 = p[7] - p[8], d910 = p[9] - p[10], d1112 = p[11] - p[12], d1314 = p[13] - p[14];
  const T ab = d78 + d910, cd = d1112 - d1314, amb = d78 - d910, cpd = d1112 + d1314;
  const T third = T(1.0 / 3.0), c24 = T(1.0 / 24.0);
  Sx = third * (p[1] - p[2]) + c24 * (ab + cd);
  Sy = third * (p[3] - p[4]) + c24 * (ab - cd);
  Sz = third * (p[5] - p[6]) + c24 * (amb + cpd);
}

// Collision of one node (Eq. 4 in the D3Q15 moment space).  f holds the
// deviations f_a - w_a rho_ref on entry and f*_a - w_a rho_ref on exit; only
// the equilibria of rows 0, 4 and 14 carry a rho_ref part (M w = (1, 0, 0, 0,
// 1, 0, ..., 0, 1/9)), so they are written in deviation form.
template <typename T>
__device__ __forceinline__ void collide(T f[kQ], T rho_ref, T Fx, T Fy, T Fz, T dS4, const Rates<T> &r) {
  // axis pairs
  const T s12 = f[1] + f[2], d12 = f[1] - f[2];
  const T s34 = f[3] + f[4], d34 = f[3] - f[4];
  const T s56 = f[5] + f[6], d56 = f[5] - f[6];
  // corner pairs -> even (count, e_x e_y, e_x e_z, e_y e_z) and odd (corner e_x,
  // e_y, e_z, e_x e_y e_z) moments by two butterfly stages
  const T s78 = f[7] + f[8], d78 = f[7] - f[8];
  const T s910 = f[9] + f[10], d910 = f[9] - f[10];
  const T s1112 = f[11] + f[12], d1112 = f[11] - f[12];
  const T s1314 = f[13] + f[14], d1314 = f[13] - f[14];
  const T u1 = s78 + s910, u2 = s1112 + s1314, v1 = s78 - s910, v2 = s1112 - s1314;
  const T m14 = u1 + u2, m7 = u1 - u2, m8 = v1 + v2, m9 = v1 - v2;
  const T U1 = d78 + d910, U2 = d1112 - d1314, V1 = d78 - d910, V2_ = d1112 + d1314;
  const T m11 = U1 + U2, m10 = U1 - U2, m12 = V1 + V2_, m13 = V1 - V2_;
  const T jx = d12 + m11, jy = d34 + m10, jz = d56 + m12;
  const T sax = s12 + s34 + s56;
  const T drho = f[0] + sax + m14;
  const T m4 = sax + T(3) * m14;
  const T m5 = T(2) * s12 - s34 - s56;
  const T m6 = s34 - s56;
  // macroscopic quantities, Eq. 6
  const T rho = rho_ref + drho;
  const T inv_rho = T(1) / rho;
  const T snu = shear_rate(r, rho);
  const T rux = jx + T(0.5) * Fx, ruy = jy + T(0.5) * Fy, ruz = jz + T(0.5) * Fz;
  const T ux = rux * inv_rho, uy = ruy * inv_rho, uz = ruz * inv_rho;
  const T qxx = rux * ux, qyy = ruy * uy, qzz = ruz * uz;  // rho u_i^2
  const T usq = qxx + qyy + qzz;
  const T third = T(1.0 / 3.0), ninth = T(1.0 / 9.0), sixth = T(1.0 / 6.0);
  const T Fux = Fx * ux, Fuy = Fy * uy, Fuz = Fz * uz;
  const T Fu = Fux + Fuy + Fuz;
  // relaxed moments
  const T mm1 = jx + Fx, mm2 = jy + Fy, mm3 = jz + Fz;
  const T mm4 = relax(m4, drho + usq, T(2) * Fu + dS4, r.se);
  const T mm5 = relax(m5, T(2) * qxx - qyy - qzz, T(2) * (T(2) * Fux - Fuy - Fuz), snu);
  const T mm6 = relax(m6, qyy - qzz, T(2) * (Fuy - Fuz), snu);
  const T mm7 = relax(m7, rux * uy, Fx * uy + Fy * ux, snu);
  const T mm8 = relax(m8, rux * uz, Fx * uz + Fz * ux, snu);
  const T mm9 = relax(m9, ruy * uz, Fy * uz + Fz * uy, snu);
  const T mm10 = relax(m10, third * ruy, third * Fy, r.sq);
  const T mm11 = relax(m11, third * rux, third * Fx, r.sq);
  const T mm12 = relax(m12, third * ruz, third * Fz, r.sq);
  const T mm13 = m13 - r.sq * m13;  // m_eq = S = 0
  const T mm14 = relax(m14, ninth * drho + T(1.0 / 18.0) * usq, T(4.0 / 9.0) * Fu, r.spi);
  // f* = M^-1 m*
  const T h = T(0.5), q = T(0.25), e8 = T(0.125);
  f[0] = drho - mm4 + T(2) * mm14;
  const T e4 = sixth * mm4, h14 = h * mm14;
  const T x_even = e4 + sixth * mm5 - h14, x_odd = h * (mm1 - mm11);
  f[1] = x_even + x_odd;
  f[2] = x_even - x_odd;
  const T e5 = T(1.0 / 12.0) * mm5, e6 = q * mm6;
  const T y_even = e4 - e5 + e6 - h14, y_odd = h * (mm2 - mm10);
  f[3] = y_even + y_odd;
  f[4] = y_even - y_odd;
  const T z_even = e4 - e5 - e6 - h14, z_odd = h * (mm3 - mm12);
  f[5] = z_even + z_odd;
  f[6] = z_even - z_odd;
  const T p1 = mm14 + mm7, p2 = mm8 + mm9, p3 = mm14 - mm7, p4 = mm8 - mm9;
  const T q1 = mm11 + mm10, q2 = mm12 + mm13, q3 = mm11 - mm10, q4 = mm12 - mm13;
  const T E78 = p1 + p2, E910 = p1 - p2, E1112 = p3 + p4, E1314 = p3 - p4;
  const T O78 = q1 + q2, O910 = q1 - q2, O1112 = q3 + q4, O1314 = q4 - q3;
  f[7] = e8 * (E78 + O78);
  f[8] = e8 * (E78 - O78);
  f[9] = e8 * (E910 + O910);
  f[10] = e8 * (E910 - O910);
  f[11] = e8 * (E1112 + O1112);
  f[12] = e8 * (E1112 - O1112);
  f[13] = e8 * (E1314 + O1314);
  f[14] = e8 * (E1314 - O1314);
}

}  // namespace q15
}  // namespace lbm
