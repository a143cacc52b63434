// Kernels of the pseudopotential MRT step and their launchers, for the D3Q19
// lattice of the paper (both operators) and its D3Q15 non-orthogonal variant
// (lbm_q15.cuh); the lattice is a template parameter Q of the one-node kernels.
//
// State layout: the stored buffer g holds, per direction a (SoA, a*N + i),
// the deviation of the post-collision population f*_a(x, t-1) from
// w_a rho_ref.  The post-streaming population of time t is pulled:
// f_a(x, t) = g_a(x - e_a) (Eq. 5).  One step is
//   psi pass:   rho(x,t) = sum_a f_a(x,t) -> psi(x)               (Eq. 6, EOS)
//   fused pass: pull f, F from psi (Eq. 15), u (Eq. 6), collide in moment
//               space (Eq. 4), store f*(x, t) at x into the other buffer.
#include <cuda_fp16.h>

#include <algorithm>

#include "lbm_device.cuh"
#include "lbm_internal.h"
#include "lbm_q15.cuh"

namespace lbm {

size_t storage_bytes(int precision) {
  return precision == kF64 ? 8 : (precision == kF32 ? 4 : 2);
}
size_t psi_elem_bytes(int precision) { return precision == kF64 ? 8 : 4; }

namespace {

template <int P> struct Types;
template <> struct Types<kF64> { using S = double; using T = double; using Psi = double; };
template <> struct Types<kF32> { using S = float; using T = float; using Psi = float; };
template <> struct Types<kF16> { using S = __half; using T = float; using Psi = float; };

// Lattice-dependent pieces of the one-node kernels.
template <int Q> struct Lat;
template <> struct Lat<19> {
  static __device__ __forceinline__ int src(const Nbhd &nb, int a) { return nb.src(a); }
  static __device__ __forceinline__ int dst(const Nbhd &nb, int a) { return nb.dst(a); }
  static __device__ __forceinline__ double w(int a) { return lattice_w(a); }
  template <typename S> static __device__ __forceinline__ typename Storage<S>::Compute load(const S *p, int a) {
    return Storage<S>::load(p, a);
  }
  template <typename S, typename T> static __device__ __forceinline__ void store(S *p, int a, T v) {
    Storage<S>::store(p, a, v);
  }
  template <typename T> static __device__ __forceinline__ void gradient(const T *p, T &Sx, T &Sy, T &Sz) {
    psi_gradient<T>(p, Sx, Sy, Sz);
  }
  static __device__ __forceinline__ void e(int a, int &x, int &y, int &z) {
    const int ex[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    const int ey[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    const int ez[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    x = ex[a];
    y = ey[a];
    z = ez[a];
  }
};
template <> struct Lat<15> {
  static __device__ __forceinline__ int src(const Nbhd &nb, int a) { return q15::src(nb, a); }
  static __device__ __forceinline__ int dst(const Nbhd &nb, int a) { return q15::dst(nb, a); }
  static __device__ __forceinline__ double w(int a) { return q15::w(a); }
  template <typename S> static __device__ __forceinline__ typename Storage<S>::Compute load(const S *p, int a) {
    return q15::Storage<S>::load(p, a);
  }
  template <typename S, typename T> static __device__ __forceinline__ void store(S *p, int a, T v) {
    q15::Storage<S>::store(p, a, v);
  }
  template <typename T> static __device__ __forceinline__ void gradient(const T *p, T &Sx, T &Sy, T &Sz) {
    q15::psi_gradient<T>(p, Sx, Sy, Sz);
  }
  static __device__ __forceinline__ void e(int a, int &x, int &y, int &z) {
    x = q15::ex(a);
    y = q15::ey(a);
    z = q15::ez(a);
  }
};

template <int Q, typename S, typename T>
__device__ __forceinline__ void pull_q(const S *__restrict__ g, int n, const Nbhd &nb, T f[Q]) {
#pragma unroll
  for (int a = 0; a < Q; ++a) f[a] = (T)Lat<Q>::load(g + (size_t)a * n + Lat<Q>::src(nb, a), a);
}

__device__ __forceinline__ bool node_of_thread(const KParams &P, int &x, int &y, int &z) {
  x = blockIdx.x * blockDim.x + threadIdx.x;
  y = blockIdx.y * blockDim.y + threadIdx.y;
  z = blockIdx.z;
  return x < P.nx && y < P.ny;
}

// ------------------------------------------------------------------ psi pass
template <int PREC, int EOS, bool DF, int Q>
__global__ void __launch_bounds__(256) psi_kernel(const typename Types<PREC>::S *__restrict__ g,
                                                  typename Types<PREC>::Psi *__restrict__ psi,
                                                  const KParams P, unsigned *__restrict__ err) {
  using S = typename Types<PREC>::S;
  using T = typename Types<PREC>::T;
  int x, y, z;
  if (!node_of_thread(P, x, y, z)) return;
  const Nbhd nb(x, y, z, P);
  T f[Q];
  pull_q<Q, S, T>(g, P.n, nb, f);
  T drho;
  if constexpr (Q == 15) {
    drho = q15::drho(f);
  } else {
    // sum in the order of the forward chain: rest + axis pairs + diagonal pairs
    const T sax = (f[1] + f[2]) + (f[3] + f[4]) + (f[5] + f[6]);
    const T sdg = ((f[7] + f[8]) + (f[9] + f[10])) + ((f[11] + f[12]) + (f[13] + f[14])) +
                  ((f[15] + f[16]) + (f[17] + f[18]));
    drho = f[0] + sax + sdg;
  }
  unsigned e = 0;
  if (DF && sizeof(T) == sizeof(float)) {
    psi[nb.self] = (typename Types<PREC>::Psi)eos_psi_f2<EOS>((float)drho, P, e);
  } else if (sizeof(T) == sizeof(float)) {
    psi[nb.self] = (typename Types<PREC>::Psi)eos_psi_d<EOS>((float)drho, P, e);
  } else {
    const double rho = P.rho_ref + (double)drho;
    const float rho_f = sizeof(T) == sizeof(double) ? (float)rho : Phys<T>::rho_ref(P) + (float)drho;
    psi[nb.self] = eos_psi<EOS, typename Types<PREC>::Psi>(rho, rho_f, P, e);
  }
  if (e) atomicOr(err, e);
}

// ------------------------------------------------------------------ fused pass
template <int PREC, int OP, bool SIGMA, int Q>
__global__ void __launch_bounds__(256) fused_kernel(const typename Types<PREC>::S *__restrict__ g_in,
                                                    typename Types<PREC>::S *__restrict__ g_out,
                                                    const typename Types<PREC>::Psi *__restrict__ psi,
                                                    const KParams P) {
  using S = typename Types<PREC>::S;
  using T = typename Types<PREC>::T;
  int x, y, z;
  if (!node_of_thread(P, x, y, z)) return;
  const Nbhd nb(x, y, z, P);
  T f[Q];
  pull_q<Q, S, T>(g_in, P.n, nb, f);
  // interaction force, Eq. 15
  T p[Q];
#pragma unroll
  for (int a = 1; a < Q; ++a) p[a] = (T)__ldg(psi + Lat<Q>::dst(nb, a));
  p[0] = (T)__ldg(psi + nb.self);
  T Sx, Sy, Sz;
  Lat<Q>::gradient(p, Sx, Sy, Sz);
  const T k = -Phys<T>::G(P) * p[0];
  const T Fx = k * Sx, Fy = k * Sy, Fz = k * Sz;
  // Eq. 16: 6 sigma |F|^2 / (psi^2 (1/s_e - 1/2)) = sigma_coef |S|^2
  const T dS4 = SIGMA ? Phys<T>::sigma_coef(P) * (Sx * Sx + Sy * Sy + Sz * Sz) : T(0);
  const Rates<T> r(P);
  if constexpr (Q == 15)
    q15::collide<T>(f, Phys<T>::rho_ref(P), Fx, Fy, Fz, dS4, r);
  else if (OP == kNonOrth)
    collide_nonorth<T>(f, Phys<T>::rho_ref(P), Fx, Fy, Fz, dS4, r);
  else
    collide_orth<T>(f, Phys<T>::rho_ref(P), Fx, Fy, Fz, dS4, r);
#pragma unroll
  for (int a = 0; a < Q; ++a) Lat<Q>::store(g_out + (size_t)a * P.n + nb.self, a, f[a]);
}

// ------------------------------------------------------------------ observables
// rho and u (Eq. 6) of the current state, in FP64 whatever the storage.
template <int PREC, int Q>
__device__ __forceinline__ void node_moments(const typename Types<PREC>::S *__restrict__ g,
                                             const typename Types<PREC>::Psi *__restrict__ psi,
                                             const KParams &P, const Nbhd &nb, double &rho,
                                             double &rux, double &ruy, double &ruz) {
  using S = typename Types<PREC>::S;
  double f[Q];
  pull_q<Q, S, double>(g, P.n, nb, f);
  double drho = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    int ex, ey, ez;
    Lat<Q>::e(a, ex, ey, ez);
    drho += f[a];
    jx += ex * f[a];
    jy += ey * f[a];
    jz += ez * f[a];
  }
  double p[Q];
#pragma unroll
  for (int a = 1; a < Q; ++a) p[a] = (double)psi[Lat<Q>::dst(nb, a)];
  p[0] = (double)psi[nb.self];
  double Sx, Sy, Sz;
  Lat<Q>::gradient(p, Sx, Sy, Sz);
  const double k = -P.G * p[0];
  rho = P.rho_ref + drho;
  rux = jx + 0.5 * k * Sx;
  ruy = jy + 0.5 * k * Sy;
  ruz = jz + 0.5 * k * Sz;
}

template <int PREC, int Q>
__global__ void moments_kernel(const typename Types<PREC>::S *__restrict__ g,
                               const typename Types<PREC>::Psi *__restrict__ psi, const KParams P,
                               double *__restrict__ rho_out, double *__restrict__ u_out) {
  int x, y, z;
  if (!node_of_thread(P, x, y, z)) return;
  const Nbhd nb(x, y, z, P);
  double rho, rux, ruy, ruz;
  node_moments<PREC, Q>(g, psi, P, nb, rho, rux, ruy, ruz);
  if (rho_out) rho_out[nb.self] = rho;
  if (u_out) {
    u_out[nb.self] = rux / rho;
    u_out[(size_t)P.n + nb.self] = ruy / rho;
    u_out[2 * (size_t)P.n + nb.self] = ruz / rho;
  }
}

// Block-partial FP64 sums of (rho, rho u) and max |u|, grid-stride over nodes,
// then one block folds the partials in a fixed order (deterministic).
template <int PREC, int Q>
__global__ void __launch_bounds__(256) diag_partial_kernel(const typename Types<PREC>::S *__restrict__ g,
                                                           const typename Types<PREC>::Psi *__restrict__ psi,
                                                           const KParams P, double *__restrict__ partials) {
  double acc[5] = {0, 0, 0, 0, 0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
    const int x = i % P.nx, yz = i / P.nx, y = yz % P.ny, z = yz / P.ny;
    const Nbhd nb(x, y, z, P);
    double rho, rux, ruy, ruz;
    node_moments<PREC, Q>(g, psi, P, nb, rho, rux, ruy, ruz);
    acc[0] += rho;
    acc[1] += rux;
    acc[2] += ruy;
    acc[3] += ruz;
    const double u = sqrt(rux * rux + ruy * ruy + ruz * ruz) / rho;
    acc[4] = (u > acc[4] || u != u) ? u : acc[4];
  }
  __shared__ double red[5][256];
#pragma unroll
  for (int k = 0; k < 5; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
#pragma unroll
      for (int k = 0; k < 4; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
      const double a = red[4][threadIdx.x], b = red[4][threadIdx.x + s];
      red[4][threadIdx.x] = (b > a || b != b) ? b : a;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < 5; ++k) partials[blockIdx.x * 5 + k] = red[k][0];
}

// max over nodes of |u(x) - u_prev(x)| (Eq. 6 velocity, FP64), folded into
// *out with an atomic max on the bit pattern (non-negative doubles order like
// their bits); u_prev is overwritten with u in FP32.
template <int PREC, int Q>
__global__ void __launch_bounds__(256) max_du_kernel(const typename Types<PREC>::S *__restrict__ g,
                                                     const typename Types<PREC>::Psi *__restrict__ psi,
                                                     const KParams P, float *__restrict__ u_prev,
                                                     unsigned long long *__restrict__ out) {
  double m = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
    const int x = i % P.nx, yz = i / P.nx, y = yz % P.ny, z = yz / P.ny;
    const Nbhd nb(x, y, z, P);
    double rho, rux, ruy, ruz;
    node_moments<PREC, Q>(g, psi, P, nb, rho, rux, ruy, ruz);
    const double u[3] = {rux / rho, ruy / rho, ruz / rho};
    double d2 = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double d = u[k] - (double)u_prev[(size_t)k * P.n + i];
      d2 += d * d;
      u_prev[(size_t)k * P.n + i] = (float)u[k];
    }
    const double d = sqrt(d2);
    m = (d > m || d != d) ? d : m;
  }
  __shared__ double red[256];
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double a = red[threadIdx.x], b = red[threadIdx.x + s];
      red[threadIdx.x] = (b > a || b != b) ? b : a;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(out, (unsigned long long)__double_as_longlong(red[0]));
}

__global__ void diag_final_kernel(const double *__restrict__ partials, int nblocks,
                                  double *__restrict__ result) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double acc[5] = {0, 0, 0, 0, 0};
  for (int b = 0; b < nblocks; ++b) {
    for (int k = 0; k < 4; ++k) acc[k] += partials[b * 5 + k];
    const double u = partials[b * 5 + 4];
    acc[4] = (u > acc[4] || u != u) ? u : acc[4];
  }
  for (int k = 0; k < 5; ++k) result[k] = acc[k];
}

// ------------------------------------------------------------------ initial state
__device__ __forceinline__ double min_image(double d, int n) {
  d = fabs(d);
  return fmin(d, (double)n - d);
}

// Eq. 59 for each droplet of the chunk; several droplets combine by maximum.
__global__ void rho_droplets_kernel(double *__restrict__ rho, const KParams P, const DropletChunk C,
                                    double W, double rho_l, double rho_v, int first) {
  int x, y, z;
  if (!node_of_thread(P, x, y, z)) return;
  const int i = x + P.nx * (y + P.ny * z);
  double best = first ? -1e300 : rho[i];
  for (int k = 0; k < C.count; ++k) {
    const double dx = min_image(x - C.cx[k], P.nx), dy = min_image(y - C.cy[k], P.ny);
    const double dz = min_image(z - C.cz[k], P.nz);
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    const double v = 0.5 * (rho_l + rho_v) - 0.5 * (rho_l - rho_v) * tanh(2.0 * (r - C.r[k]) / W);
    best = fmax(best, v);
  }
  rho[i] = best;
}

// Liquid slab between planes lo and hi across one axis (Sec. IV D).
__global__ void rho_slab_kernel(double *__restrict__ rho, const KParams P, int axis, double lo,
                                double hi, double W, double rho_l, double rho_v) {
  int x, y, z;
  if (!node_of_thread(P, x, y, z)) return;
  const double c = axis == 0 ? x : (axis == 1 ? y : z);
  rho[x + P.nx * (y + P.ny * z)] =
      rho_v + 0.5 * (rho_l - rho_v) * (tanh(2.0 * (c - lo) / W) - tanh(2.0 * (c - hi) / W));
}

// f_a(x, 0) = w_a rho0(x): store g_a(y) = w_a (rho0(y + e_a) - rho_ref).
template <int PREC, int Q>
__global__ void state_from_rho_kernel(const double *__restrict__ rho, typename Types<PREC>::S *__restrict__ g,
                                      const KParams P) {
  using S = typename Types<PREC>::S;
  int x, y, z;
  if (!node_of_thread(P, x, y, z)) return;
  const Nbhd nb(x, y, z, P);
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    const double v = Lat<Q>::w(a) * (rho[Lat<Q>::dst(nb, a)] - P.rho_ref);
    Lat<Q>::store(g + (size_t)a * P.n + nb.self, a, (typename Types<PREC>::T)v);
  }
}

// out[(a - a_lo) N + i] = f_a(x_i, t) for a in [a_lo, a_hi).
template <int PREC, int Q>
__global__ void get_populations_kernel(const typename Types<PREC>::S *__restrict__ g, double *__restrict__ out,
                                       const KParams P, int a_lo, int a_hi) {
  using S = typename Types<PREC>::S;
  int x, y, z;
  if (!node_of_thread(P, x, y, z)) return;
  const Nbhd nb(x, y, z, P);
#pragma unroll
  for (int a = 0; a < Q; ++a)
    if (a >= a_lo && a < a_hi)
      out[(size_t)(a - a_lo) * P.n + nb.self] =
          Lat<Q>::w(a) * P.rho_ref + (double)Lat<Q>::load(g + (size_t)a * P.n + Lat<Q>::src(nb, a), a);
}

// Reverse of the above: g_a(y) = f_a(y + e_a) - w_a rho_ref.
template <int PREC, int Q>
__global__ void set_populations_kernel(const double *__restrict__ f, typename Types<PREC>::S *__restrict__ g,
                                       const KParams P, int a_lo, int a_hi) {
  using S = typename Types<PREC>::S;
  int x, y, z;
  if (!node_of_thread(P, x, y, z)) return;
  const Nbhd nb(x, y, z, P);
#pragma unroll
  for (int a = 0; a < Q; ++a)
    if (a >= a_lo && a < a_hi) {
      const double v = f[(size_t)(a - a_lo) * P.n + Lat<Q>::dst(nb, a)] - Lat<Q>::w(a) * P.rho_ref;
      Lat<Q>::store(g + (size_t)a * P.n + nb.self, a, (typename Types<PREC>::T)v);
    }
}

dim3 node_grid(const KParams &P, const Launch &L) {
  return dim3((P.nx + L.bx - 1) / L.bx, (P.ny + L.by - 1) / L.by, P.nz);
}

template <int PREC, bool DF, int Q>
cudaError_t psi_dispatch(const KParams &P, const void *g, void *psi, unsigned *err, const Launch &L) {
  using S = typename Types<PREC>::S;
  using Psi = typename Types<PREC>::Psi;
  const dim3 grid = node_grid(P, L), block(L.bx, L.by);
  switch (P.eos) {
    case kEosCS:
      psi_kernel<PREC, kEosCS, DF, Q><<<grid, block, 0, L.stream>>>((const S *)g, (Psi *)psi, P, err);
      break;
    case kEosExp:
      psi_kernel<PREC, kEosExp, DF, Q><<<grid, block, 0, L.stream>>>((const S *)g, (Psi *)psi, P, err);
      break;
    default:
      psi_kernel<PREC, kEosNone, DF, Q><<<grid, block, 0, L.stream>>>((const S *)g, (Psi *)psi, P, err);
      break;
  }
  return cudaGetLastError();
}

template <int PREC, int OP, int Q>
cudaError_t fused_dispatch(const KParams &P, bool sigma, const void *g_in, void *g_out, const void *psi,
                           const Launch &L) {
  using S = typename Types<PREC>::S;
  using Psi = typename Types<PREC>::Psi;
  const dim3 grid = node_grid(P, L), block(L.bx, L.by);
  if (sigma)
    fused_kernel<PREC, OP, true, Q><<<grid, block, 0, L.stream>>>((const S *)g_in, (S *)g_out, (const Psi *)psi, P);
  else
    fused_kernel<PREC, OP, false, Q><<<grid, block, 0, L.stream>>>((const S *)g_in, (S *)g_out, (const Psi *)psi, P);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_psi(const KParams &P, int precision, const void *g, void *psi, unsigned *err,
                       const Launch &L, bool df) {
  if (P.q == 15) {
    if (pair_supported(P, precision)) return launch_psi_pair(P, precision, g, psi, err, L, df);
    switch (precision) {
      case kF64: return psi_dispatch<kF64, false, 15>(P, g, psi, err, L);
      case kF32:
        return df ? psi_dispatch<kF32, true, 15>(P, g, psi, err, L) : psi_dispatch<kF32, false, 15>(P, g, psi, err, L);
      default:
        return df ? psi_dispatch<kF16, true, 15>(P, g, psi, err, L) : psi_dispatch<kF16, false, 15>(P, g, psi, err, L);
    }
  }
  switch (precision) {
    case kF64: return psi_dispatch<kF64, false, 19>(P, g, psi, err, L);
    case kF32:
      if (pair_supported(P, precision)) return launch_psi_pair(P, precision, g, psi, err, L, df);
      return df ? psi_dispatch<kF32, true, 19>(P, g, psi, err, L) : psi_dispatch<kF32, false, 19>(P, g, psi, err, L);
    default:
      if (pair_supported(P, precision)) return launch_psi_pair(P, precision, g, psi, err, L, df);
      return df ? psi_dispatch<kF16, true, 19>(P, g, psi, err, L) : psi_dispatch<kF16, false, 19>(P, g, psi, err, L);
  }
}

cudaError_t launch_fused(const KParams &P, int precision, int op, bool sigma, const void *g_in, void *g_out,
                         const void *psi, const Launch &L) {
  if (P.q == 15) {
    if (pair_supported(P, precision)) return launch_fused_pair(P, precision, op, sigma, g_in, g_out, psi, L);
    switch (precision) {
      case kF64: return fused_dispatch<kF64, kNonOrth, 15>(P, sigma, g_in, g_out, psi, L);
      case kF32: return fused_dispatch<kF32, kNonOrth, 15>(P, sigma, g_in, g_out, psi, L);
      default: return fused_dispatch<kF16, kNonOrth, 15>(P, sigma, g_in, g_out, psi, L);
    }
  }
  if (pair_supported(P, precision)) return launch_fused_pair(P, precision, op, sigma, g_in, g_out, psi, L);
  if (op == kNonOrth) {
    switch (precision) {
      case kF64: return fused_dispatch<kF64, kNonOrth, 19>(P, sigma, g_in, g_out, psi, L);
      case kF32: return fused_dispatch<kF32, kNonOrth, 19>(P, sigma, g_in, g_out, psi, L);
      default: return fused_dispatch<kF16, kNonOrth, 19>(P, sigma, g_in, g_out, psi, L);
    }
  }
  switch (precision) {
    case kF64: return fused_dispatch<kF64, kOrth, 19>(P, sigma, g_in, g_out, psi, L);
    case kF32: return fused_dispatch<kF32, kOrth, 19>(P, sigma, g_in, g_out, psi, L);
    default: return fused_dispatch<kF16, kOrth, 19>(P, sigma, g_in, g_out, psi, L);
  }
}

// CALL with PR = the precision and QQ = the lattice, both compile-time constants.
#define LBM_PREC_SWITCH_Q(precision, QV, CALL)                     \
  switch (precision) {                                             \
    case kF64: { constexpr int PR = kF64, QQ = QV; CALL; } break; \
    case kF32: { constexpr int PR = kF32, QQ = QV; CALL; } break; \
    default: { constexpr int PR = kF16, QQ = QV; CALL; } break;   \
  }
#define LBM_PREC_SWITCH(precision, CALL)                         \
  if (P.q == 15) {                                               \
    LBM_PREC_SWITCH_Q(precision, 15, CALL)                       \
  } else {                                                       \
    LBM_PREC_SWITCH_Q(precision, 19, CALL)                       \
  }

cudaError_t launch_moments(const KParams &P, int precision, const void *g, const void *psi, double *rho,
                           double *u, const Launch &L) {
  const dim3 grid = node_grid(P, L), block(L.bx, L.by);
  LBM_PREC_SWITCH(precision, (moments_kernel<PR, QQ><<<grid, block, 0, L.stream>>>(
                                 (const typename Types<PR>::S *)g, (const typename Types<PR>::Psi *)psi, P, rho, u)));
  return cudaGetLastError();
}

cudaError_t launch_diag(const KParams &P, int precision, const void *g, const void *psi, double *partials,
                        double *result, const Launch &L) {
  LBM_PREC_SWITCH(precision, (diag_partial_kernel<PR, QQ><<<kReduceBlocks, 256, 0, L.stream>>>(
                                 (const typename Types<PR>::S *)g, (const typename Types<PR>::Psi *)psi, P, partials)));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  diag_final_kernel<<<1, 32, 0, L.stream>>>(partials, kReduceBlocks, result);
  return cudaGetLastError();
}

cudaError_t launch_max_du(const KParams &P, int precision, const void *g, const void *psi, float *u_prev,
                          double *out, const Launch &L) {
  const int blocks = (int)std::min<long long>(4 * 152, ((long long)P.n + 255) / 256);
  LBM_PREC_SWITCH(precision, (max_du_kernel<PR, QQ><<<blocks, 256, 0, L.stream>>>(
                                 (const typename Types<PR>::S *)g, (const typename Types<PR>::Psi *)psi, P, u_prev,
                                 (unsigned long long *)out)));
  return cudaGetLastError();
}

cudaError_t launch_rho_droplets(const KParams &P, double *rho, const DropletChunk &chunk, double W,
                                double rho_l, double rho_v, bool first, const Launch &L) {
  rho_droplets_kernel<<<node_grid(P, L), dim3(L.bx, L.by), 0, L.stream>>>(rho, P, chunk, W, rho_l, rho_v,
                                                                           first ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_rho_slab(const KParams &P, double *rho, int axis, double lo, double hi, double W,
                            double rho_l, double rho_v, const Launch &L) {
  rho_slab_kernel<<<node_grid(P, L), dim3(L.bx, L.by), 0, L.stream>>>(rho, P, axis, lo, hi, W, rho_l, rho_v);
  return cudaGetLastError();
}

cudaError_t launch_state_from_rho(const KParams &P, int precision, const double *rho, void *g, const Launch &L) {
  const dim3 grid = node_grid(P, L), block(L.bx, L.by);
  LBM_PREC_SWITCH(precision, (state_from_rho_kernel<PR, QQ><<<grid, block, 0, L.stream>>>(
                                 rho, (typename Types<PR>::S *)g, P)));
  return cudaGetLastError();
}

cudaError_t launch_get_populations(const KParams &P, int precision, const void *g, double *out, int a_lo,
                                   int a_hi, const Launch &L) {
  const dim3 grid = node_grid(P, L), block(L.bx, L.by);
  LBM_PREC_SWITCH(precision, (get_populations_kernel<PR, QQ><<<grid, block, 0, L.stream>>>(
                                 (const typename Types<PR>::S *)g, out, P, a_lo, a_hi)));
  return cudaGetLastError();
}

cudaError_t launch_set_populations(const KParams &P, int precision, const double *f, void *g, int a_lo,
                                   int a_hi, const Launch &L) {
  const dim3 grid = node_grid(P, L), block(L.bx, L.by);
  LBM_PREC_SWITCH(precision, (set_populations_kernel<PR, QQ><<<grid, block, 0, L.stream>>>(
                                 f, (typename Types<PR>::S *)g, P, a_lo, a_hi)));
  return cudaGetLastError();
}

}  // namespace lbm
