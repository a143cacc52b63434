// Device-side building blocks of the D3Q19 pseudopotential MRT step:
// lattice addressing, population storage, the equation of state, the
// interaction force and the two collision operators written as sparse
// add/sub chains (the transformation matrices are never stored).
//
// Directions follow Eq. 2: 0 rest; 1,2 = +-x; 3,4 = +-y; 5,6 = +-z;
// 7..10 = (1,1,0),(-1,-1,0),(1,-1,0),(-1,1,0); 11..14 = (1,0,1),(-1,0,-1),
// (1,0,-1),(-1,0,1); 15..18 = (0,1,1),(0,-1,-1),(0,1,-1),(0,-1,1).
#pragma once

#include <cuda_fp16.h>
#include <math.h>

#include "lbm_debug.cuh"
#include "lbm_internal.h"

namespace lbm {

// ------------------------------------------------------------------ addressing
// Periodic neighbours of a node and the row offsets (y, z part of the index)
// of the nine (y', z') combinations a D3Q19 stencil touches.
struct Nbhd {
  int x, xm, xp;                                   // x, x-1, x+1 (wrapped)
  int r00, rm0, rp0, r0m, r0p, rmm, rpp, rmp, rpm;  // nx*(y' + ny*z')
  int self;

  __device__ __forceinline__ Nbhd(int x_, int y, int z, const KParams &P) {
    x_ = LBM_IDX(x_, P.nx);  // debug build: the node must lie in the box
    y = LBM_IDX(y, P.ny);
    z = LBM_IDX(z, P.nz);
    x = x_;
    xm = x_ == 0 ? P.nx - 1 : x_ - 1;
    xp = x_ == P.nx - 1 ? 0 : x_ + 1;
    const int ym = y == 0 ? P.ny - 1 : y - 1, yp = y == P.ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? P.nz - 1 : z - 1, zp = z == P.nz - 1 ? 0 : z + 1;
    const int nx = P.nx, nxy = P.nx * P.ny;
    const int z0 = z * nxy, zM = zm * nxy, zP = zp * nxy;
    r00 = y * nx + z0;  rm0 = ym * nx + z0;  rp0 = yp * nx + z0;
    r0m = y * nx + zM;  r0p = y * nx + zP;
    rmm = ym * nx + zM; rpp = yp * nx + zP; rmp = ym * nx + zP; rpm = yp * nx + zM;
    self = r00 + x_;
  }

  // Node x - e_a: where population a of node x comes from (pull streaming, Eq. 5).
  __device__ __forceinline__ int src(int a) const {
    switch (a) {
      case 0: return r00 + x;
      case 1: return r00 + xm;   case 2: return r00 + xp;
      case 3: return rm0 + x;    case 4: return rp0 + x;
      case 5: return r0m + x;    case 6: return r0p + x;
      case 7: return rm0 + xm;   case 8: return rp0 + xp;
      case 9: return rp0 + xm;   case 10: return rm0 + xp;
      case 11: return r0m + xm;  case 12: return r0p + xp;
      case 13: return r0p + xm;  case 14: return r0m + xp;
      case 15: return rmm + x;   case 16: return rpp + x;
      case 17: return rmp + x;   default: return rpm + x;
    }
  }

  // Node x + e_a: the neighbour read by the interaction force (Eq. 15).
  __device__ __forceinline__ int dst(int a) const {
    switch (a) {
      case 0: return r00 + x;
      case 1: return r00 + xp;   case 2: return r00 + xm;
      case 3: return rp0 + x;    case 4: return rm0 + x;
      case 5: return r0p + x;    case 6: return r0m + x;
      case 7: return rp0 + xp;   case 8: return rm0 + xm;
      case 9: return rm0 + xp;   case 10: return rp0 + xm;
      case 11: return r0p + xp;  case 12: return r0m + xm;
      case 13: return r0m + xp;  case 14: return r0p + xm;
      case 15: return rpp + x;   case 16: return rmm + x;
      case 17: return rpm + x;   default: return rmp + x;
    }
  }
};

// Lattice weights of the rest state, f_a = w_a rho (= M^-1 m_eq(rho, 0) for
// both operators).
__device__ __forceinline__ constexpr double lattice_w(int a) {
  return a == 0 ? 1.0 / 3.0 : (a < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
}
__device__ __forceinline__ constexpr float lattice_inv_w(int a) {
  return a == 0 ? 3.0f : (a < 7 ? 18.0f : 36.0f);
}

// ------------------------------------------------------------------ storage
// A stored population is the deviation f_a - w_a rho_ref; the FP16 form stores
// it divided by w_a so every direction uses the same range.
template <typename S> struct Storage;

template <> struct Storage<double> {
  using Compute = double;
  static __device__ __forceinline__ double decode(double v, int a) { (void)a; return v; }
  static __device__ __forceinline__ double load(const double *p, int a) { (void)a; return __ldg(p); }
  static __device__ __forceinline__ void store(double *p, int a, double v) { (void)a; *p = v; }
};

template <> struct Storage<float> {
  using Compute = float;
  static __device__ __forceinline__ float decode(float v, int a) { (void)a; return v; }
  static __device__ __forceinline__ float load(const float *p, int a) { (void)a; return __ldg(p); }
  static __device__ __forceinline__ void store(float *p, int a, float v) { (void)a; *p = v; }
};

template <> struct Storage<__half> {
  using Compute = float;
  static __device__ __forceinline__ float decode(__half v, int a) { return __half2float(v) * (float)lattice_w(a); }
  static __device__ __forceinline__ float load(const __half *p, int a) {
    return __half2float(__ldg(p)) * (float)lattice_w(a);
  }
  static __device__ __forceinline__ void store(__half *p, int a, float v) {
    *p = __float2half_rn(v * lattice_inv_w(a));
  }
};


// ------------------------------------------------------------------ EOS
// psi(rho): square-root form sqrt(2 (p_EOS - rho/3) / G) with the
// Carnahan-Starling p_EOS of Eq. 58, or psi0 exp(-rho0/rho) (Sec. II B).
// With eta = b rho/4, num = 1 + eta + eta^2 - eta^3 and den = (1 - eta)^3 the
// radicand is X / den, X = (2/G) rho (RT num - (a rho + 1/3) den): a quintic in
// rho with no division, evaluated by Horner's rule from host-made coefficients
// (KParams::q0..q4), always in FP64 (the repulsive and attractive parts of
// p_EOS cancel there).  psi = X rsqrt(X den); the FP32-psi forms take den and
// the root in FP32, the precision psi is stored in.
// Outside the domain (rho <= 0 or not finite, b rho/4 >= 1, negative radicand)
// it flags the error and returns NaN: the state is never clamped.
// rho_f is rho rounded to FP32 (used for the domain checks and the final root).
template <int EOS, typename PsiT>
__device__ __forceinline__ PsiT eos_psi(double rho, float rho_f, const KParams &P, unsigned &err) {
  const PsiT nan = (PsiT)__longlong_as_double(0x7ff8000000000000LL);
  if (EOS == kEosNone) return PsiT(0);
  if (!isfinite(rho_f)) { err |= kErrNonFinite; return nan; }
  if (!(rho_f > 0.0f)) { err |= kErrEosDomain; return nan; }
  if (EOS == kEosExp) return (PsiT)(P.psi0 * exp(-P.rho0 / rho));
  if (!(rho_f < P.f_rho_max)) { err |= kErrEosDomain; return nan; }
  const double X = rho * fma(fma(fma(fma(P.q4, rho, P.q3), rho, P.q2), rho, P.q1), rho, P.q0);
  if (sizeof(PsiT) == sizeof(double)) {
    if (!(X >= 0.0)) { err |= kErrEosDomain; return nan; }
    if (X == 0.0) return PsiT(0);
    const double one_m = fma(-P.b4, rho, 1.0);
    return (PsiT)(X * rsqrt(X * (one_m * one_m * one_m)));
  }
  const float xf = (float)X;
  if (!(xf >= 0.0f)) { err |= kErrEosDomain; return nan; }
  if (xf == 0.0f) return PsiT(0);
  const float one_m = fmaf(-P.fb4, rho_f, 1.0f);
  return (PsiT)(xf * rsqrtf(xf * (one_m * one_m * one_m)));
}

// FP32 -> FP64 widening and FP64 -> FP32 rounding (to nearest, ties to even)
// done on the integer units: GB300 issues two FP64 instructions per SM and
// clock, conversions included, and the EOS below is bound by that rate, while
// the integer units are idle.  Both are exact bit manipulations of IEEE 754
// binary32 / binary64 (bias 127 / 1023, 23 / 52 fraction bits), so the results
// equal the conversion instructions'; values outside the range handled (zero
// and subnormal inputs, results outside the normal FP32 range) take the
// conversion instruction.
__device__ __forceinline__ double widen_f32(float v) {
  const unsigned u = __float_as_uint(v), ex = u & 0x7f800000u;
  if (ex == 0x7f800000u || (ex == 0u && (u << 1) != 0u)) return (double)v;  // inf, nan, subnormal
  // sign, exponent + (1023 - 127), top 20 fraction bits; the last 3 fraction bits open the low word (a zero
  // keeps its sign and nothing else)
  const unsigned hi = ex ? (u & 0x80000000u) | (((u >> 3) & 0x0fffffffu) + 0x38000000u) : (u & 0x80000000u);
  return __hiloint2double((int)hi, (int)(u << 29));
}

__device__ __forceinline__ float narrow_f64(double v) {
  const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
  const unsigned E = (hi >> 20) & 0x7ffu;
  if (E < 897u || E > 1150u) return (float)v;  // FP32 exponent E - 896 outside 1..254
  // sign, E - 896, the top 23 of the 52 fraction bits; then round on the 29 dropped bits
  unsigned r = (hi & 0x80000000u) | (((hi & 0x7fffffffu) - (896u << 20)) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1fffffffu;
  r += (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ? 1u : 0u;  // a carry moves into the exponent
  return __uint_as_float(r);
}

// psi in FP32 from d = rho - rho_ref (the FP32-arithmetic forms): the radicand
// X as a quintic in d, Horner in FP64 from host-made coefficients (KParams::c),
// five FMA and no separate rho_ref + d, one FP64 operation fewer than the
// quintic in rho; checks and the final root as in eos_psi's FP32-psi path.
template <int EOS, bool ICVT = true>
__device__ __forceinline__ float eos_psi_d(float d, const KParams &P, unsigned &err) {
  const float nan = __int_as_float(0x7fc00000);
  if (EOS == kEosNone) return 0.f;
  const float rho_f = P.frho_ref + d;
  if (!isfinite(rho_f)) { err |= kErrNonFinite; return nan; }
  if (!(rho_f > 0.0f)) { err |= kErrEosDomain; return nan; }
  if (EOS == kEosExp) return (float)(P.psi0 * exp(-P.rho0 / (P.rho_ref + (double)d)));
  if (!(rho_f < P.f_rho_max)) { err |= kErrEosDomain; return nan; }
  const double x = ICVT ? widen_f32(d) : (double)d;
  const double X = fma(fma(fma(fma(fma(P.c[5], x, P.c[4]), x, P.c[3]), x, P.c[2]), x, P.c[1]), x, P.c[0]);
  const float xf = ICVT ? narrow_f64(X) : (float)X;
  if (!(xf >= 0.0f)) { err |= kErrEosDomain; return nan; }
  if (xf == 0.0f) return 0.f;
  const float one_m = fmaf(-P.fb4, rho_f, 1.0f);
  return xf * rsqrtf(xf * (one_m * one_m * one_m));
}

// Compensated FP32 arithmetic on unevaluated sums hi + lo of two floats
// (error-free transformations: Knuth's TwoSum, Dekker's Fast2Sum, the exact
// product error by FMA).  The intrinsics keep the compiler from contracting or
// reassociating the steps.
struct F2 {
  float h, l;
};
__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ F2 fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
  const F2 s = two_sum(a.h, b.h);
  return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ F2 f2_mul(F2 a, F2 b) {
  const float p = __fmul_rn(a.h, b.h);
  const float e = __fmaf_rn(a.h, b.h, -p);
  return fast_two_sum(p, __fadd_rn(e, __fadd_rn(__fmul_rn(a.h, b.l), __fmul_rn(a.l, b.h))));
}

// psi in FP32 with the radicand X evaluated in compensated FP32 pairs instead
// of FP64 (about 44 significant bits; GB300 has two FP64 lanes per SM against
// 128 FP32).  rho = rho_ref + drho is formed exactly.  The checks and the final
// root are those of eos_psi's FP32-psi path, so psi agrees with it wherever the
// pair's leading float equals the FP64 radicand rounded to FP32.
template <int EOS>
__device__ __forceinline__ float eos_psi_f2(float drho, const KParams &P, unsigned &err) {
  const float nan = __int_as_float(0x7fc00000);
  if (EOS == kEosNone) return 0.f;
  const float rho_f = P.frho_ref + drho;
  if (!isfinite(rho_f)) { err |= kErrNonFinite; return nan; }
  if (!(rho_f > 0.0f)) { err |= kErrEosDomain; return nan; }
  if (EOS == kEosExp) return (float)(P.psi0 * exp(-P.rho0 / (P.rho_ref + (double)drho)));
  if (!(rho_f < P.f_rho_max)) { err |= kErrEosDomain; return nan; }
  F2 rho = two_sum(P.rr_h, drho);
  rho = fast_two_sum(rho.h, __fadd_rn(rho.l, P.rr_l));
  F2 acc = {P.qh[4], P.ql[4]};
#pragma unroll
  for (int k = 3; k >= 0; --k) acc = f2_add(f2_mul(acc, rho), F2{P.qh[k], P.ql[k]});
  const float xf = f2_mul(acc, rho).h;
  if (!(xf >= 0.0f)) { err |= kErrEosDomain; return nan; }
  if (xf == 0.0f) return 0.f;
  const float one_m = fmaf(-P.fb4, rho_f, 1.0f);
  return xf * rsqrtf(xf * (one_m * one_m * one_m));
}

// ------------------------------------------------------------------ force
// S = sum_a w_a psi(x + e_a) e_a with w = 1/6 (axes), 1/12 (diagonals);
// F = -G psi(x) S (Eq. 15).  p[a] = psi(x + e_a).
template <typename T>
__device__ __forceinline__ void psi_gradient(const T p[19], T &Sx, T &Sy, T &Sz) {
  const T d78 = p[7] - p[8], d910 = p[9] - p[10], d1112 = p[11] - p[12];
  const T d1314 = p[13] - p[14], d1516 = p[15] - p[16], d1718 = p[17] - p[18];
  const T sixth = T(1.0 / 6.0), twelfth = T(1.0 / 12.0);
  Sx = sixth * (p[1] - p[2]) + twelfth * ((d78 + d910) + (d1112 + d1314));
  Sy = sixth * (p[3] - p[4]) + twelfth * ((d78 - d910) + (d1516 + d1718));
  Sz = sixth * (p[5] - p[6]) + twelfth * ((d1112 - d1314) + (d1516 - d1718));
}

// ------------------------------------------------------------------ packed pairs
// V2 holds one FP32 quantity of two x-adjacent nodes; its arithmetic issues one
// packed FP32 instruction (add, multiply, fused multiply-add on float2, sm_100
// family) for both nodes.  A product stays unevaluated (V2Mul) until it is
// added to something, so "c + a * b" becomes one packed FMA: the contraction
// the compiler applies to the scalar FP32 code.  The instructions carry an
// explicit round-to-nearest modifier, which rules out any further contraction
// by the compiler: every kernel built on V2 rounds exactly where the source
// says.  Division and the shear-rate evaluation act lane by lane.  The
// collision templates run on V2 unchanged.
__device__ __forceinline__ float2 pk_add(float2 a, float2 b) {
  float2 d;
  asm("{.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 pk_mul(float2 a, float2 b) {
  float2 d;
  asm("{.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 pk_fma(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\t"
      "mov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
struct V2 {
  float2 v;
  V2() = default;
  __device__ __forceinline__ V2(float2 a) : v(a) {}
  __device__ __forceinline__ V2(float a, float b) : v(make_float2(a, b)) {}
  __device__ __forceinline__ explicit V2(double c) : v(make_float2((float)c, (float)c)) {}
};
__device__ __forceinline__ V2 v2neg(V2 a) { return V2(-a.v.x, -a.v.y); }
__device__ __forceinline__ V2 v2fma(V2 a, V2 b, V2 c) { return pk_fma(a.v, b.v, c.v); }
struct V2Mul {
  V2 a, b;
  __device__ __forceinline__ operator V2() const { return pk_mul(a.v, b.v); }
};
__device__ __forceinline__ V2 operator+(V2 a, V2 b) { return pk_add(a.v, b.v); }
__device__ __forceinline__ V2 operator-(V2 a, V2 b) { return pk_add(a.v, v2neg(b).v); }
__device__ __forceinline__ V2 operator-(V2 a) { return v2neg(a); }
__device__ __forceinline__ V2Mul operator*(V2 a, V2 b) { return {a, b}; }
__device__ __forceinline__ V2 operator/(V2 a, V2 b) { return V2(a.v.x / b.v.x, a.v.y / b.v.y); }
__device__ __forceinline__ V2 operator+(V2Mul p, V2 c) { return v2fma(p.a, p.b, c); }
__device__ __forceinline__ V2 operator+(V2 c, V2Mul p) { return v2fma(p.a, p.b, c); }
__device__ __forceinline__ V2 operator-(V2 c, V2Mul p) { return v2fma(v2neg(p.a), p.b, c); }
__device__ __forceinline__ V2 operator-(V2Mul p, V2 c) { return v2fma(p.a, p.b, v2neg(c)); }
__device__ __forceinline__ V2 operator+(V2Mul p, V2Mul q) { return v2fma(p.a, p.b, V2(q)); }
__device__ __forceinline__ V2 operator-(V2Mul p, V2Mul q) { return v2fma(v2neg(q.a), q.b, V2(p)); }
__device__ __forceinline__ V2Mul operator-(V2Mul p) { return {v2neg(p.a), p.b}; }
__device__ __forceinline__ V2Mul operator*(V2Mul p, V2 c) { return {V2(p), c}; }
__device__ __forceinline__ V2Mul operator*(V2 c, V2Mul p) { return {c, V2(p)}; }

// ------------------------------------------------------------------ collision
template <typename T> struct Rates;
template <> struct Rates<double> {
  double se, snu, sq, spi, seps, sm;
  bool varnu;
  double nu_v, rho_v, nu_slope, nu_lo, nu_hi;
  __device__ __forceinline__ explicit Rates(const KParams &P)
      : se(P.s_e), snu(P.s_nu), sq(P.s_q), spi(P.s_pi), seps(P.s_eps), sm(P.s_m), varnu(P.varnu != 0),
        nu_v(P.nu_v), rho_v(P.rho_v_nu), nu_slope(P.nu_slope), nu_lo(P.nu_lo), nu_hi(P.nu_hi) {}
};
template <> struct Rates<float> {
  float se, snu, sq, spi, seps, sm;
  bool varnu;
  float nu_v, rho_v, nu_slope, nu_lo, nu_hi;
  __device__ __forceinline__ explicit Rates(const KParams &P)
      : se(P.fs_e), snu(P.fs_nu), sq(P.fs_q), spi(P.fs_pi), seps(P.fs_eps), sm(P.fs_m), varnu(P.varnu != 0),
        nu_v(P.fnu_v), rho_v(P.frho_v_nu), nu_slope(P.fnu_slope), nu_lo(P.fnu_lo), nu_hi(P.fnu_hi) {}
};

template <> struct Rates<V2> {
  Rates<float> s;  // scalar copy, for the density-dependent shear rate
  V2 se, snu, sq, spi, seps, sm;
  __device__ __forceinline__ explicit Rates(const KParams &P)
      : s(P), se(s.se), snu(s.snu), sq(s.sq), spi(s.spi), seps(s.seps), sm(s.sm) {}
};

// Shear rate at density rho: constant, or 1 / (3 nu(rho) + 1/2) with nu linear
// in rho between the phases and clamped to the two phase values.
template <typename T>
__device__ __forceinline__ T shear_rate(const Rates<T> &r, T rho) {
  if (!r.varnu) return r.snu;
  T nu = r.nu_v + (rho - r.rho_v) * r.nu_slope;
  nu = nu < r.nu_lo ? r.nu_lo : (nu > r.nu_hi ? r.nu_hi : nu);
  return T(1) / (T(3) * nu + T(0.5));
}
__device__ __forceinline__ V2 shear_rate(const Rates<V2> &r, V2 rho) {
  if (!r.s.varnu) return r.snu;
  return V2(shear_rate(r.s, rho.v.x), shear_rate(r.s, rho.v.y));
}

// Parameters in the arithmetic type of a kernel (FP32 kernels read the float copies).
template <typename T> struct Phys;
template <> struct Phys<double> {
  static __device__ __forceinline__ double G(const KParams &P) { return P.G; }
  static __device__ __forceinline__ double rho_ref(const KParams &P) { return P.rho_ref; }
  static __device__ __forceinline__ double sigma_coef(const KParams &P) { return P.sigma_coef; }
};
template <> struct Phys<float> {
  static __device__ __forceinline__ float G(const KParams &P) { return P.fG; }
  static __device__ __forceinline__ float rho_ref(const KParams &P) { return P.frho_ref; }
  static __device__ __forceinline__ float sigma_coef(const KParams &P) { return P.fsigma_coef; }
};

// relax one moment: m* = m - s (m - m_eq) + (1 - s/2) S   (Eq. 4)
template <typename T>
__device__ __forceinline__ T relax(T m, T meq, T S, T s) {
  return m + s * (meq - m) + (T(1) - T(0.5) * s) * S;
}
__device__ __forceinline__ V2 relax(V2 m, V2 meq, V2 S, V2 s) {
  return m + s * (meq - m) + (V2(1.0) - V2(0.5) * s) * S;
}

// Non-orthogonal operator: forward chains of Eq. 12, equilibria Eq. 13,
// forcing Eq. 14 (+ Eq. 16 via dS4), inverse chains of App. A.
// f holds the deviations f_a - w_a rho_ref on entry and f*_a - w_a rho_ref on
// exit; the chains act on deviations directly because M and M^-1 are linear
// and only m_eq carries the rho_ref part (rho_ref M w = rho_ref (1,0,0,0,1,0..0,1/9,1/9,1/9)).
template <typename T>
__device__ __forceinline__ void collide_nonorth(T f[19], T rho_ref, T Fx, T Fy, T Fz, T dS4,
                                                const Rates<T> &r) {
  // opposite-pair sums and differences
  const T s12 = f[1] + f[2], d12 = f[1] - f[2];
  const T s34 = f[3] + f[4], d34 = f[3] - f[4];
  const T s56 = f[5] + f[6], d56 = f[5] - f[6];
  const T s78 = f[7] + f[8], d78 = f[7] - f[8];
  const T s910 = f[9] + f[10], d910 = f[9] - f[10];
  const T s1112 = f[11] + f[12], d1112 = f[11] - f[12];
  const T s1314 = f[13] + f[14], d1314 = f[13] - f[14];
  const T s1516 = f[15] + f[16], d1516 = f[15] - f[16];
  const T s1718 = f[17] + f[18], d1718 = f[17] - f[18];
  // m = M f (Eq. 12), in deviation form (m - rho_ref M w)
  const T m16 = s78 + s910, m17 = s1112 + s1314, m18 = s1516 + s1718;
  const T m7 = s78 - s910, m8 = s1112 - s1314, m9 = s1516 - s1718;
  const T m10 = d78 - d910, m11 = d78 + d910;
  const T m12 = d1112 - d1314, m13 = d1112 + d1314;
  const T m14 = d1516 - d1718, m15 = d1516 + d1718;
  const T jx = d12 + m11 + m13;
  const T jy = d34 + m10 + m15;
  const T jz = d56 + m12 + m14;
  const T sax = s12 + s34 + s56;
  const T sdg = m16 + m17 + m18;
  const T drho = f[0] + sax + sdg;
  const T m4 = sax + T(2) * sdg;
  const T m5 = T(2) * s12 - s34 - s56 + m16 + m17 - T(2) * m18;
  const T m6 = s34 - s56 + m16 - m17;
  // macroscopic quantities, Eq. 6
  const T rho = rho_ref + drho;
  const T inv_rho = T(1) / rho;
  const T snu = shear_rate(r, rho);
  const T rux = jx + T(0.5) * Fx, ruy = jy + T(0.5) * Fy, ruz = jz + T(0.5) * Fz;
  const T ux = rux * inv_rho, uy = ruy * inv_rho, uz = ruz * inv_rho;
  const T qxx = rux * ux, qyy = ruy * uy, qzz = ruz * uz;  // rho u_i^2
  const T usq = qxx + qyy + qzz;
  const T third = T(1.0 / 3.0), ninth = T(1.0 / 9.0), sixth = T(1.0 / 6.0);
  // forcing products
  const T Fux = Fx * ux, Fuy = Fy * uy, Fuz = Fz * uz;
  // relaxed moments (Eq. 4 with Eqs. 11, 13, 14)
  const T mm1 = jx + Fx, mm2 = jy + Fy, mm3 = jz + Fz;
  const T mm4 = relax(m4, drho + usq, T(2) * (Fux + Fuy + Fuz) + dS4, r.se);
  const T mm5 = relax(m5, T(2) * qxx - qyy - qzz, T(2) * (T(2) * Fux - Fuy - Fuz), snu);
  const T mm6 = relax(m6, qyy - qzz, T(2) * (Fuy - Fuz), snu);
  const T mm7 = relax(m7, rux * uy, Fx * uy + Fy * ux, snu);
  const T mm8 = relax(m8, rux * uz, Fx * uz + Fz * ux, snu);
  const T mm9 = relax(m9, ruy * uz, Fy * uz + Fz * uy, snu);
  const T mm10 = relax(m10, third * ruy, third * Fy, r.sq);
  const T mm11 = relax(m11, third * rux, third * Fx, r.sq);
  const T mm12 = relax(m12, third * ruz, third * Fz, r.sq);
  const T mm13 = relax(m13, third * rux, third * Fx, r.sq);
  const T mm14 = relax(m14, third * ruz, third * Fz, r.sq);
  const T mm15 = relax(m15, third * ruy, third * Fy, r.sq);
  const T phi = ninth * drho - sixth * usq;  // phi + (rho - rho_ref)/9 part of Eq. 13
  const T mm16 = relax(m16, phi + third * (qxx + qyy), T(2) * third * (Fux + Fuy), r.spi);
  const T mm17 = relax(m17, phi + third * (qxx + qzz), T(2) * third * (Fux + Fuz), r.spi);
  const T mm18 = relax(m18, phi + third * (qyy + qzz), T(2) * third * (Fuy + Fuz), r.spi);
  // f* = M^-1 m* (App. A)
  const T h = T(0.5), q = T(0.25);
  f[0] = drho - mm4 + mm16 + mm17 + mm18;
  const T e4 = sixth * mm4;
  const T ex_odd = h * (mm1 - mm11 - mm13);
  const T ex_even = e4 + sixth * mm5 - h * (mm16 + mm17);
  f[1] = ex_even + ex_odd;
  f[2] = ex_even - ex_odd;
  const T e5 = T(1.0 / 12.0) * mm5, e6 = q * mm6;
  const T ey_odd = h * (mm2 - mm10 - mm15);
  const T ey_even = e4 - e5 + e6 - h * (mm16 + mm18);
  f[3] = ey_even + ey_odd;
  f[4] = ey_even - ey_odd;
  const T ez_odd = h * (mm3 - mm12 - mm14);
  const T ez_even = e4 - e5 - e6 - h * (mm17 + mm18);
  f[5] = ez_even + ez_odd;
  f[6] = ez_even - ez_odd;
  const T a7 = mm7 + mm16, b7 = mm7 - mm16, c10 = mm10 + mm11, d10 = mm10 - mm11;
  f[7] = q * (a7 + c10);
  f[8] = q * (a7 - c10);
  f[9] = q * (-b7 - d10);
  f[10] = q * (-b7 + d10);
  const T a11 = mm8 + mm17, b11 = mm8 - mm17, c12 = mm12 + mm13, k12 = mm12 - mm13;
  f[11] = q * (a11 + c12);
  f[12] = q * (a11 - c12);
  f[13] = q * (-b11 - k12);
  f[14] = q * (-b11 + k12);
  const T a15 = mm9 + mm18, b15 = mm9 - mm18, c14 = mm14 + mm15, d14 = mm14 - mm15;
  f[15] = q * (a15 + c14);
  f[16] = q * (a15 - c14);
  f[17] = q * (-b15 - d14);
  f[18] = q * (-b15 + d14);
}

// Orthogonal operator (d'Humieres et al. D3Q19 basis at the Eq. 2 ordering):
// m = M_o f, m_eq = M_o f_eq, S = M_o G (Guo), f* = M_o^T diag(1/|row|^2) m*.
// The Eq. 16 term enters as dS4 * (0, 19, -16, 0, ...), its image in this basis.
template <typename T>
__device__ __forceinline__ void collide_orth(T f[19], T rho_ref, T Fx, T Fy, T Fz, T dS4,
                                             const Rates<T> &r) {
  const T s12 = f[1] + f[2], d12 = f[1] - f[2];
  const T s34 = f[3] + f[4], d34 = f[3] - f[4];
  const T s56 = f[5] + f[6], d56 = f[5] - f[6];
  const T s78 = f[7] + f[8], d78 = f[7] - f[8];
  const T s910 = f[9] + f[10], d910 = f[9] - f[10];
  const T s1112 = f[11] + f[12], d1112 = f[11] - f[12];
  const T s1314 = f[13] + f[14], d1314 = f[13] - f[14];
  const T s1516 = f[15] + f[16], d1516 = f[15] - f[16];
  const T s1718 = f[17] + f[18], d1718 = f[17] - f[18];
  const T sxy = s78 + s910, sxz = s1112 + s1314, syz = s1516 + s1718;
  const T A = s12 + s34 + s56, B = sxy + sxz + syz;
  // forward transform M_o f; on deviations it gives m - rho_ref (1, -11, 3, 0, ...)
  const T drho = f[0] + A + B;
  const T m1 = T(-30) * f[0] - T(11) * A + T(8) * B;
  const T m2 = T(12) * f[0] - T(4) * A + B;
  const T dx = d78 + d910 + d1112 + d1314;
  const T dy = d78 - d910 + d1516 + d1718;
  const T dz = d1112 - d1314 + d1516 - d1718;
  const T jx = d12 + dx, jy = d34 + dy, jz = d56 + dz;
  const T m4 = dx - T(4) * d12, m6 = dy - T(4) * d34, m8 = dz - T(4) * d56;
  const T sxyz = sxy + sxz;
  const T m9 = T(2) * s12 - s34 - s56 + sxyz - T(2) * syz;
  const T m10 = T(-4) * s12 + T(2) * (s34 + s56) + sxyz - T(2) * syz;
  const T m11 = s34 - s56 + sxy - sxz;
  const T m12 = T(-2) * s34 + T(2) * s56 + sxy - sxz;
  const T m13 = s78 - s910, m14 = s1516 - s1718, m15 = s1112 - s1314;
  const T m16 = d78 + d910 - d1112 - d1314;
  const T m17 = d1516 + d1718 - d78 + d910;
  const T m18 = d1112 - d1314 - d1516 + d1718;
  // macroscopic quantities, Eq. 6
  const T rho = rho_ref + drho;
  const T inv_rho = T(1) / rho;
  const T snu = shear_rate(r, rho);
  const T rux = jx + T(0.5) * Fx, ruy = jy + T(0.5) * Fy, ruz = jz + T(0.5) * Fz;
  const T ux = rux * inv_rho, uy = ruy * inv_rho, uz = ruz * inv_rho;
  const T qxx = rux * ux, qyy = ruy * uy, qzz = ruz * uz;
  const T usq = qxx + qyy + qzz;
  const T Fux = Fx * ux, Fuy = Fy * uy, Fuz = Fz * uz;
  const T Fu = Fux + Fuy + Fuz;
  const T two3 = T(2.0 / 3.0);
  // relaxed moments
  const T pxx = T(2) * qxx - qyy - qzz, pww = qyy - qzz;
  const T Sxx = T(2) * Fux - Fuy - Fuz, Sww = Fuy - Fuz;
  const T mm1 = relax(m1, T(-11) * drho + T(19) * usq, T(38) * Fu + T(19) * dS4, r.se);
  const T mm2 = relax(m2, T(3) * drho - T(5.5) * usq, T(-11) * Fu - T(16) * dS4, r.seps);
  const T mm3 = jx + Fx, mm5 = jy + Fy, mm7 = jz + Fz;
  const T mm4 = relax(m4, -two3 * rux, -two3 * Fx, r.sq);
  const T mm6 = relax(m6, -two3 * ruy, -two3 * Fy, r.sq);
  const T mm8 = relax(m8, -two3 * ruz, -two3 * Fz, r.sq);
  const T mm9 = relax(m9, pxx, T(2) * Sxx, snu);
  const T mm10 = relax(m10, T(-0.5) * pxx, -Sxx, r.spi);
  const T mm11 = relax(m11, pww, T(2) * Sww, snu);
  const T mm12 = relax(m12, T(-0.5) * pww, -Sww, r.spi);
  const T mm13 = relax(m13, rux * uy, Fx * uy + Fy * ux, snu);
  const T mm14 = relax(m14, ruy * uz, Fy * uz + Fz * uy, snu);
  const T mm15 = relax(m15, rux * uz, Fx * uz + Fz * ux, snu);
  const T sm1 = T(1) - r.sm;
  const T mm16 = sm1 * m16, mm17 = sm1 * m17, mm18 = sm1 * m18;
  // inverse: f*_a = sum_k M_o[k][a] m*_k / |row k|^2
  const T n0 = drho * T(1.0 / 19.0), n1 = mm1 * T(1.0 / 2394.0), n2 = mm2 * T(1.0 / 252.0);
  const T n3 = mm3 * T(0.1), n4 = mm4 * T(0.025), n5 = mm5 * T(0.1), n6 = mm6 * T(0.025);
  const T n7 = mm7 * T(0.1), n8 = mm8 * T(0.025);
  const T n9 = mm9 * T(1.0 / 36.0), n10 = mm10 * T(1.0 / 72.0);
  const T n11 = mm11 * T(1.0 / 12.0), n12 = mm12 * T(1.0 / 24.0);
  const T n13 = mm13 * T(0.25), n14 = mm14 * T(0.25), n15 = mm15 * T(0.25);
  const T n16 = mm16 * T(0.125), n17 = mm17 * T(0.125), n18 = mm18 * T(0.125);
  f[0] = n0 - T(30) * n1 + T(12) * n2;
  const T Ca = n0 - T(11) * n1 - T(4) * n2;
  const T xo = n3 - T(4) * n4, yo = n5 - T(4) * n6, zo = n7 - T(4) * n8;
  const T p9 = T(2) * n9 - T(4) * n10;        // axis x: 3pxx, 3pi_xx
  const T q9 = -n9 + T(2) * n10;              // axes y, z
  const T w11 = n11 - T(2) * n12;             // axis y: +, axis z: -
  f[1] = Ca + xo + p9;
  f[2] = Ca - xo + p9;
  f[3] = Ca + yo + q9 + w11;
  f[4] = Ca - yo + q9 + w11;
  f[5] = Ca + zo + q9 - w11;
  f[6] = Ca - zo + q9 - w11;
  const T Cd = n0 + T(8) * n1 + n2;
  const T Exy = Cd + n9 + n10 + n11 + n12;
  const T Exz = Cd + n9 + n10 - n11 - n12;
  const T Eyz = Cd - T(2) * (n9 + n10);
  const T X = n3 + n4, Y = n5 + n6, Z = n7 + n8;
  // xy diagonals 7..10: signs of (p_xy, m_x, m_y) are (+,+,-), (+,-,+), (-,+,+), (-,-,-)
  {
    const T pp = X + Y, pm = X - Y, a = n16 - n17, c = n16 + n17;
    f[7] = Exy + pp + n13 + a;
    f[8] = Exy - pp + n13 - a;
    f[9] = Exy + pm - n13 + c;
    f[10] = Exy - pm - n13 - c;
  }
  // xz diagonals 11..14: signs of (p_xz, m_x, m_z) are (+,-,+), (+,+,-), (-,-,-), (-,+,+)
  {
    const T pp = X + Z, pm = X - Z, a = n18 - n16, c = n16 + n18;
    f[11] = Exz + pp + n15 + a;
    f[12] = Exz - pp + n15 - a;
    f[13] = Exz + pm - n15 - c;
    f[14] = Exz - pm - n15 + c;
  }
  // yz diagonals 15..18: signs of (p_yz, m_y, m_z) are (+,+,-), (+,-,+), (-,+,+), (-,-,-)
  {
    const T pp = Y + Z, pm = Y - Z, a = n17 - n18, c = n17 + n18;
    f[15] = Eyz + pp + n14 + a;
    f[16] = Eyz - pp + n14 - a;
    f[17] = Eyz + pm - n14 + c;
    f[18] = Eyz - pm - n14 - c;
  }
}

}  // namespace lbm
