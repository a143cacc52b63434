// Index bounds checks of the debug build (compiled with -DLBM_BOUNDS_CHECK).
//
// LBM_IDX(i, n) is i in the normal build.  In the debug build it checks
// 0 <= i < n; an index outside that range is replaced by 0 (so the access
// that follows stays inside the buffer) and a bit is set in this translation
// unit's device error word.  Nothing traps.  Every translation unit that
// includes this header registers a reader of its word with the context code,
// which folds the words into lbm_check / lbm_batch_check (LBM_ERR_BOUNDS).
#pragma once

#include <cuda_runtime.h>

#ifdef LBM_BOUNDS_CHECK

namespace lbm {
namespace dbg {

static __device__ unsigned bounds_err;  // one per translation unit

__device__ __forceinline__ int checked(int i, int n) {
  if ((unsigned)i >= (unsigned)n) {
    atomicOr(&bounds_err, 1u);
    return 0;
  }
  return i;
}

using Reader = unsigned (*)();
bool register_reader(Reader r);  // lbm_api.cu

// Read and clear this translation unit's word (synchronous).
static unsigned read_and_clear() {
  unsigned v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, bounds_err, sizeof v) != cudaSuccess) return 0;
  cudaMemcpyToSymbol(bounds_err, &zero, sizeof zero);
  return v;
}
static const bool registered = register_reader(read_and_clear);

}  // namespace dbg
}  // namespace lbm

#define LBM_IDX(i, n) ::lbm::dbg::checked((i), (n))

#else

#define LBM_IDX(i, n) (i)

#endif
