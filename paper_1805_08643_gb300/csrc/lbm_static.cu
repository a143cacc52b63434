// lbm_step_static: one FP64 time step that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA graph is
// being captured, hosts whose device memory is owned by another allocator or
// arena, and real-time loops that must not allocate or risk an allocation
// failure.  This entry point serves them.  The caller passes the populations
// in and out; the only scratch the step needs (psi, one value per node) lives
// in the fixed-size array below, which every GPU that loads the library keeps
// until the process exits.
#include <cuda_runtime.h>

#include "../../include/lbm.h"
#include "lbm_device.cuh"
#include "lbm_internal.h"

// Largest box this entry point accepts: 2^21 nodes (128^3); 16 MiB of psi.
#define LBM_STATIC_MAX_NODES (1 << 21)

static __device__ __align__(256) double lbm_static_psi[LBM_STATIC_MAX_NODES];

// The parts of lbm_ctx this entry point reads (lbm_api.cu owns the struct).
namespace lbm {
bool ctx_params(const lbm_ctx *c, KParams *P, int *precision, int *op, bool *sigma_on, cudaStream_t *stream);
}

namespace {

using lbm::KParams;
using lbm::Nbhd;

// psi from the unshifted populations f_a(x, t) (public layout, absolute values).
template <int EOS>
__global__ void static_psi_kernel(const double *__restrict__ f, double *__restrict__ psi, const KParams P) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
  if (x >= P.nx || y >= P.ny) return;
  const int i = x + P.nx * (y + P.ny * z);
  double rho = 0.0;
#pragma unroll
  for (int a = 0; a < 19; ++a) rho += f[(size_t)a * P.n + i];
  unsigned e = 0;
  psi[i] = lbm::eos_psi<EOS, double>(rho, (float)rho, P, e);  // out of the EOS domain: NaN, which reaches f_out
}

// Collide f_a(x, t) and push f*_a(x, t) to f_out at x + e_a (Eq. 5).
template <int OP, bool SIGMA>
__global__ void static_fused_kernel(const double *__restrict__ f_in, double *__restrict__ f_out,
                                    const double *__restrict__ psi, const KParams P) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
  if (x >= P.nx || y >= P.ny) return;
  const Nbhd nb(x, y, z, P);
  double f[19], p[19];
#pragma unroll
  for (int a = 0; a < 19; ++a) f[a] = f_in[(size_t)a * P.n + nb.self];
#pragma unroll
  for (int a = 1; a < 19; ++a) p[a] = psi[nb.dst(a)];
  p[0] = psi[nb.self];
  double Sx, Sy, Sz;
  lbm::psi_gradient<double>(p, Sx, Sy, Sz);
  const double Fx = -P.G * p[0] * Sx, Fy = -P.G * p[0] * Sy, Fz = -P.G * p[0] * Sz;
  const double dS4 = SIGMA ? P.sigma_coef * (Sx * Sx + Sy * Sy + Sz * Sz) : 0.0;
  const lbm::Rates<double> r(P);
  if (OP == lbm::kNonOrth)
    lbm::collide_nonorth<double>(f, 0.0, Fx, Fy, Fz, dS4, r);
  else
    lbm::collide_orth<double>(f, 0.0, Fx, Fy, Fz, dS4, r);
#pragma unroll
  for (int a = 0; a < 19; ++a) f_out[(size_t)a * P.n + nb.dst(a)] = f[a];
}

// Device address of lbm_static_psi, looked up on the first call on each device
// (with that device current) and kept for the life of the process.  A
// cudaDeviceReset frees the module that holds the array, so the kept address
// is stale after one: this entry point is not for processes that reset a
// device they have called it on.
constexpr int kMaxDevices = 64;
double *g_psi_addr[kMaxDevices] = {nullptr};

cudaError_t static_psi_address(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (!g_psi_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, lbm_static_psi);
    if (e != cudaSuccess) return e;
    g_psi_addr[dev] = (double *)p;
  }
  *out = g_psi_addr[dev];
  return cudaSuccess;
}

// Launch through cudaLaunchKernel, whose return value is this launch's own
// status: an unrelated error left earlier on the calling thread is neither
// reported as this step's failure nor cleared.
template <typename K>
cudaError_t launch(K kernel, dim3 grid, dim3 block, cudaStream_t stream, void **args) {
  return cudaLaunchKernel((const void *)kernel, grid, block, args, 0, stream);
}

}  // namespace

extern "C" lbm_status lbm_step_static(const lbm_ctx *ctx, const double *f_in, double *f_out) {
  if (!ctx || !f_in || !f_out || f_in == f_out) return LBM_ERR_ARG;
  KParams P;
  int precision = 0, op = 0;
  bool sigma_on = false;
  cudaStream_t stream = nullptr;
  if (!lbm::ctx_params(ctx, &P, &precision, &op, &sigma_on, &stream)) return LBM_ERR_ARG;
  if (precision != LBM_F64) return LBM_ERR_ARG;                 // FP64 populations only
  if (P.q != 19) return LBM_ERR_ARG;                            // D3Q19 kernels only
  if ((long long)P.n > LBM_STATIC_MAX_NODES) return LBM_ERR_ARG;  // beyond the static psi array
  P.rho_ref = 0.0;  // f_in / f_out hold absolute populations
  double *psi = nullptr;
  if (static_psi_address(&psi) != cudaSuccess) return LBM_ERR_CUDA;
  const dim3 block(32, 4), grid((P.nx + 31) / 32, (P.ny + 3) / 4, P.nz);
  void *psi_args[] = {(void *)&f_in, (void *)&psi, (void *)&P};
  cudaError_t e;
  switch (P.eos) {
    case lbm::kEosCS: e = launch(static_psi_kernel<lbm::kEosCS>, grid, block, stream, psi_args); break;
    case lbm::kEosExp: e = launch(static_psi_kernel<lbm::kEosExp>, grid, block, stream, psi_args); break;
    default: e = launch(static_psi_kernel<lbm::kEosNone>, grid, block, stream, psi_args); break;
  }
  if (e != cudaSuccess) return LBM_ERR_CUDA;
  const double *psi_c = psi;
  void *fused_args[] = {(void *)&f_in, (void *)&f_out, (void *)&psi_c, (void *)&P};
  if (op == lbm::kNonOrth)
    e = sigma_on ? launch(static_fused_kernel<lbm::kNonOrth, true>, grid, block, stream, fused_args)
                 : launch(static_fused_kernel<lbm::kNonOrth, false>, grid, block, stream, fused_args);
  else
    e = sigma_on ? launch(static_fused_kernel<lbm::kOrth, true>, grid, block, stream, fused_args)
                 : launch(static_fused_kernel<lbm::kOrth, false>, grid, block, stream, fused_args);
  return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}
