// Lattice diagnostics without any allocation: the same reduction as
// wrc_diagnostics (energy, enstrophy, palinstrophy, circulation of a
// reconstructed vorticity lattice and its streamfunction), with its scratch
// -- one row of partial sums per block and the last-block counter -- in a
// file-scope device array instead of memory the library allocates.
//
// Some callers cannot allocate device memory: code that runs while a stream
// is being captured into a CUDA graph (an allocation there either fails or
// becomes part of the graph), host frameworks that own the whole device
// memory budget through their own pool and forbid other allocators, and
// real-time loops where cudaMalloc/cudaFree would synchronise the device at
// unpredictable moments.  They pass their own input and output buffers and
// this entry point uses only the fixed array below.
#include <mutex>

#include "../../include/wrc.h"
#include "kernels.h"

namespace wrc {
namespace {

// One partial row of 4 sums per block of the reduction grid (capped at
// kMaxBlocks blocks), then the counter of finished blocks: 39 KB per device,
// held by every device that loads the library until the process exits.
constexpr int kNoAllocPartials = kMaxBlocks * 4;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocPartials + 4];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Scale the raw lattice sums to E = h^2/2 sum |U|^2, Z = h^2/2 sum R^2,
// P = h^2/2 sum |grad R|^2, circulation = h^2 sum R (as wrc_diagnostics).
__global__ void k_noalloc_scale(double* out, double h2) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const double s0 = out[0], s1 = out[1], s2 = out[2], s3 = out[3];
        out[0] = 0.5 * h2 * s2;
        out[1] = 0.5 * h2 * s1;
        out[2] = 0.5 * h2 * s3;
        out[3] = h2 * s0;
    }
}

}  // namespace
}  // namespace wrc

using namespace wrc;

extern "C" wrc_status wrc_lattice_diagnostics_noalloc(const double* omega_lattice, const double* psi_lattice,
                                                      int32_t NJ, double* out, void* cuda_stream) {
    if (!omega_lattice || !psi_lattice || !out) return WRC_ERR_ARG;
    if (NJ < 8 || NJ > WRC_MAX_NJ || (NJ & (NJ - 1))) return WRC_ERR_ARG;   // beyond the stated maximum
    const cudaStream_t s = (cudaStream_t)cuda_stream;
    // the array is looked up for the device the stream belongs to, which
    // must be the current one (a kernel is launched on the current device)
    int dev = 0, sdev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return WRC_ERR_CUDA;
    if (cudaStreamGetDevice(s, &sdev) != cudaSuccess) return WRC_ERR_ARG;
    if (sdev != dev) return WRC_ERR_ARG;
    double* scratch = nullptr;
    {
        // set-up, once per device (with that device current): the device
        // address of the array; the host-side symbol is only a stand-in
        std::lock_guard<std::mutex> lk(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return WRC_ERR_CUDA;
            g_noalloc_ptr[dev] = (double*)p;
        }
        scratch = g_noalloc_ptr[dev];
    }
    unsigned* counter = (unsigned*)(scratch + kNoAllocPartials);
    // the counter must start at zero; the partial rows are overwritten
    if (cudaMemsetAsync(counter, 0, sizeof(unsigned), s) != cudaSuccess) return WRC_ERR_CUDA;
    Geom g{};
    g.NJ = NJ;
    int L = 0;
    while ((1 << L) < NJ) ++L;
    g.L = L;
    g.J = 0;
    g.mask = NJ - 1;
    g.h = 2.0 * 3.141592653589793238462643383279502884 / NJ;
    g.P = 2;   // the order-4 stencils
    if (launch_diag<double>(omega_lattice, psi_lattice, scratch, counter, out, g, s) != cudaSuccess) return WRC_ERR_CUDA;
    double h2 = g.h * g.h;
    void* args[] = {(void*)&out, (void*)&h2};
    if (cudaLaunchKernel((const void*)k_noalloc_scale, dim3(1), dim3(1), args, 0, s) != cudaSuccess)
        return WRC_ERR_CUDA;
    note_launch();
    return WRC_OK;
}
