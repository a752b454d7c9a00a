// piccs_reg_normal_noalloc: the regularisation normal operator D^T diag(omega) D z
// (+ lambda^2 z for PIPLE) and its energy sum omega |Dz|^2, for callers that
// cannot allocate device memory.
//
// Who needs it: code that runs inside a host application which owns all of the
// GPU's memory through its own pool with a hard cap (a plugin must not take
// memory behind the pool's back), and latency-critical loops in which a
// cudaMalloc/cudaFree would synchronise the whole device.  Such callers cannot
// create a piccs_ctx (piccs_create allocates the workspace), so this entry
// point takes plain sizes and caller-owned buffers, like the rest of the ABI,
// and keeps its only scratch -- the per-CTA FP64 partial sums of the energy --
// in a fixed array in this file.
//
// The scratch array is a file-scope __device__ array: every GPU that loads
// this library holds it (32 KiB) until the process exits.  In host code its
// name is only a host-side stand-in for the device symbol, so the device
// address is looked up once per device with cudaGetSymbolAddress (on the first
// call made with that device current) and passed to the kernels.  The address
// is kept for the life of the process, so the entry point must not be used on
// a device after a cudaDeviceReset of it (the module, and with it the array,
// may then be loaded at another address).
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/piccs.h"
#include "internal.h"

namespace {

constexpr int kScratchDoubles = 4096;  // maximum per-CTA partial sums
constexpr int kMaxDevices = 64;
// the stencil grid never exceeds kStencilMaxBlocks CTAs, whatever the volume
static_assert(piccs::kStencilMaxBlocks <= kScratchDoubles,
              "the partial-sum scratch must hold one entry per stencil CTA");

__device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_mutex;
double *g_scratch_ptr[kMaxDevices] = {};

int fail(int code, const char *msg)
{
    piccs::set_thread_error(msg);  // read back with piccs_last_error(NULL)
    return code;
}

}  // namespace

extern "C" int piccs_reg_normal_noalloc(int nx, int ny, int nz, const float *d_omega,
                                        float lambda2_piple, const float *d_z, float *d_out,
                                        double *d_rho, void *cuda_stream)
{
    if (nx <= 0 || ny <= 0 || nz <= 0) return fail(PICCS_EINVAL, "volume size must be positive");
    const long long M = (long long)nx * ny * nz;
    if (M > 2147483647LL) return fail(PICCS_EINVAL, "nx*ny*nz exceeds 2^31-1 voxels");
    if (!d_omega || !d_z || !d_out || !d_rho) return fail(PICCS_EINVAL, "NULL buffer");
    if (!std::isfinite(lambda2_piple) || lambda2_piple < 0.f)
        return fail(PICCS_EINVAL, "lambda2_piple must be finite and >= 0");
    const int blocks = piccs::stencil_blocks(M);  // <= kStencilMaxBlocks (static_assert above)

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(PICCS_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(PICCS_EINVAL, "device ordinal beyond 63");
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return fail(PICCS_ECUDA, cudaGetErrorString(e));
            g_scratch_ptr[dev] = static_cast<double *>(p);
        }
        scratch = g_scratch_ptr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // every CTA overwrites its own partial before the one-CTA sum reads the
    // first `blocks` entries, so nothing has to be cleared between calls
    e = piccs::launch_reg_normal(piccs::VolDims{nx, ny, nz}, d_z, d_omega, lambda2_piple, d_out,
                                 scratch, st);
    if (e == cudaSuccess) e = piccs::launch_sum_partials(scratch, blocks, d_rho, st);
    if (e != cudaSuccess) return fail(PICCS_ECUDA, cudaGetErrorString(e));
    return PICCS_OK;
}
