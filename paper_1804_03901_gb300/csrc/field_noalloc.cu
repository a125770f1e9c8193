// field_noalloc.cu -- allocation-free variant of the stand-alone spectral
// Poisson solve (avl_field_solve_noalloc in include/avl.h).
//
// Some callers cannot allocate device memory at the point where they need a
// field solve: a host program whose GPU memory is already fully reserved by
// another allocator (a framework's caching allocator, a fixed memory budget),
// or a time-critical loop that must not pay for cudaMalloc / cudaFree, which
// synchronise the device.  For them the transform tables (the only scratch
// the solve needs) live in one file-scope device array.  The CUDA runtime
// places it on a GPU together with this file's kernels when the first call
// there loads the module (lazy loading), and it stays until the process
// exits; callers make that first call before they reserve the rest of the
// GPU's memory and before any stream capture.
#include <cuda_runtime.h>
#include <math.h>

#include "avl_internal.cuh"

namespace avl {

// largest grid the fixed scratch serves: the largest nx whose solve fits one
// block's 200 KiB of shared memory (16 nx + 32 bytes without staged tables);
// power-of-two grids stop at 8192 below it
constexpr int NOALLOC_MAX_NX = 12798;
// twiddles exp(-2 pi i k / nx) (nx complex) followed by cP kappa / K^2 (nx/2 + 1)
constexpr size_t NOALLOC_TW_BYTES = (size_t)NOALLOC_MAX_NX * sizeof(double2);
constexpr size_t NOALLOC_BYTES = NOALLOC_TW_BYTES + ((size_t)NOALLOC_MAX_NX / 2 + 1) * sizeof(double);

static __device__ __align__(256) unsigned char g_field_scratch[NOALLOC_BYTES];

// tables computed on the device, same formulas as the host tables of
// avl_field_solve (Eq. 6a-c, sinc(y) = sin(y)/y; Eq. 5 without softening)
__global__ void k_noalloc_tables(int nx, double L, double cP, int softening)
{
    // device code may name the array directly
    double2* tw = reinterpret_cast<double2*>(g_field_scratch);
    double* gm = reinterpret_cast<double*>(g_field_scratch + NOALLOC_TW_BYTES);
    const double dx = L / nx;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nx; k += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)k / (double)nx, &s, &c);
        tw[k] = make_double2(c, -s);
        if (k <= nx / 2) {
            double g = 0.0;
            if (k > 0 && 2 * k != nx) {
                const double kk = 2.0 * M_PI * (double)k / L;
                double kappa = kk, K2 = kk * kk;
                if (softening) {
                    const double y1 = kk * dx, y2 = 0.5 * kk * dx;
                    kappa = kk * (sin(y1) / y1);
                    K2 = kk * kk * (sin(y2) / y2) * (sin(y2) / y2);
                }
                g = cP * kappa / K2;
            }
            gm[k] = g;
        }
    }
}

namespace {
// the device address of the array on the current device (its name in host
// code is only a host-side stand-in).  Looked up on every call: after the
// first call has loaded the module on a device the lookup allocates nothing,
// and a context reset that reloads the module at another address is
// followed.
cudaError_t scratch_address(void** out)
{
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_field_scratch);
    if (e) return e;
    *out = p;
    return cudaSuccess;
}
}  // namespace

}  // namespace avl

extern avl_status avl_noalloc_fail(avl_status st, const char* msg);

extern "C" avl_status avl_field_solve_noalloc(int32_t nx, double L, double poisson_const, int32_t softening,
                                              const double* rho, double* E, void* cuda_stream)
{
    using namespace avl;
    if (nx < 4 || nx > NOALLOC_MAX_NX)
        return avl_noalloc_fail(AVL_EINVAL,
                                "nx must be in [4, 12798] for the allocation-free field solve (the largest grid "
                                "one block's shared memory solves)");
    if (!(L > 0) || !(poisson_const > 0) || !isfinite(L) || !isfinite(poisson_const))
        return avl_noalloc_fail(AVL_EINVAL, "L and poisson_const must be positive and finite");
    if (softening != 0 && softening != 1) return avl_noalloc_fail(AVL_EINVAL, "softening must be 0 or 1");
    if (!rho || !E) return avl_noalloc_fail(AVL_EINVAL, "rho or E is NULL");
    if (poisson_smem_bytes(nx) > 200 * 1024) return avl_noalloc_fail(AVL_EINVAL, "nx too large for one block");
    void* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e) return avl_noalloc_fail(AVL_ECUDA, cudaGetErrorString(e));
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const double2* tw = static_cast<const double2*>(base);
    const double* gm = reinterpret_cast<const double*>(static_cast<unsigned char*>(base) + NOALLOC_TW_BYTES);
    k_noalloc_tables<<<(nx + 255) / 256, 256, 0, st>>>(nx, L, poisson_const, softening);
    e = cudaGetLastError();
    if (!e) e = launch_poisson(rho, E, nx, tw, gm, st);
    if (e) return avl_noalloc_fail(AVL_ECUDA, cudaGetErrorString(e));
    return AVL_OK;
}
