// Krylov kernels of DD order 2p = 6 (single-run and batched, FP64 and the
// mixed mode), compiled in a translation unit of their own.
#include "krylov_impl.cuh"

namespace wrc {
template struct KrylovKernels<double, 3>;
template struct KrylovKernels<float, 3>;
}  // namespace wrc
