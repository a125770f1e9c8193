// k_moments.cu -- output quantities of Sec. 3.4.2 that the time step does not
// use, formed on demand from the stored reconstruction: the velocity moments
// of one species (charge, current density per velocity component, trace of
// the second moment) and the residual charge of the field solve.
#include <math.h>

#include <algorithm>

#include "avl_internal.cuh"

namespace avl {

// out[m][x] += q dvol sum_cells w_m(v) f(x, v) with w = 1, v_x, (v_y, v_z),
// |v|^2 (midpoint rule over the cell-centred velocity grid, as Eq. 14).
// Block: 32 columns x 8 row lanes over a range of velocity cells; FP64 sums.
template <typename T>
__global__ void __launch_bounds__(256) k_moments(const StepArgs* __restrict__ A, int s, int rows_per_block,
                                                 double* __restrict__ out)
{
    __shared__ double red[5][8][32];
    const SpDev& sp = A->sp[s];
    const int nx = sp.nx, nvf = sp.nvflat, nd = sp.nvdim;
    const int col = threadIdx.x & 31, lr = threadIdx.x >> 5;
    const int x = blockIdx.x * 32 + col;
    const int j0 = blockIdx.y * rows_per_block, j1 = min(nvf, j0 + rows_per_block);
    const T* f = reinterpret_cast<const T*>(sp.fgrid);
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (x < nx) {
        for (int j = j0 + lr; j < j1; j += 8) {
            // velocity-cell centre of row j (1d3v rows are [vz][vy][vx])
            double v[3] = {0.0, 0.0, 0.0};
            int r = j;
            for (int d = 0; d < nd; ++d) {
                const int k = r % sp.nv[d];
                r /= sp.nv[d];
                v[d] = sp.vmin[d] + (k + 0.5) * sp.dv[d];
            }
            const double fv = (double)f[(size_t)j * nx + x];
            acc[0] += fv;
            acc[1] += v[0] * fv;
            acc[2] += v[1] * fv;
            acc[3] += v[2] * fv;
            acc[4] += (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) * fv;
        }
    }
    for (int m = 0; m < 5; ++m) red[m][lr][col] = acc[m];
    __syncthreads();
    if (lr == 0 && x < nx) {
        double dvol = 1.0;
        for (int d = 0; d < nd; ++d) dvol *= sp.dv[d];
        const double c = sp.q * dvol;
        const int nmom = 2 + nd;
        for (int m = 0; m < nmom; ++m) {
            const int src = m == nmom - 1 ? 4 : m;   // rho, j_x, (j_y, j_z), M2
            double t = 0.0;
            for (int k = 0; k < 8; ++k) t += red[src][k][col];
            atomicAdd(out + (size_t)m * nx + x, c * t);
        }
    }
}

// drho_i = rho_i - (E_{i+1} - E_{i-1}) / (2 dx cP), periodic
__global__ void k_residual(const StepArgs* __restrict__ A, double* __restrict__ out)
{
    const FieldDev& fd = A->fd;
    const int nx = fd.nx;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nx; i += gridDim.x * blockDim.x) {
        const int ip = i + 1 == nx ? 0 : i + 1, im = i == 0 ? nx - 1 : i - 1;
        out[i] = fd.rho[i] - (fd.E64[ip] - fd.E64[im]) / (2.0 * fd.dx * fd.cP);
    }
}

cudaError_t launch_moments(const StepArgs& h, const StepArgs* d, int s, double* out, cudaStream_t st)
{
    const SpDev& sp = h.sp[s];
    const int nmom = 2 + sp.nvdim;
    cudaError_t e = cudaMemsetAsync(out, 0, (size_t)nmom * sp.nx * 8, st);
    if (e) return e;
    const int xb = (sp.nx + 31) / 32;
    const int groups = std::max(1, std::min(sp.nvflat / 8 + 1, (4 * 152 + xb - 1) / xb));
    const int rows = (sp.nvflat + groups - 1) / groups;
    dim3 grid(xb, (sp.nvflat + rows - 1) / rows);
    if (h.prec == AVL_FP32)
        k_moments<float><<<grid, 256, 0, st>>>(d, s, rows, out);
    else
        k_moments<double><<<grid, 256, 0, st>>>(d, s, rows, out);
    return cudaGetLastError();
}

cudaError_t launch_residual(const StepArgs& h, const StepArgs* d, double* out, cudaStream_t st)
{
    k_residual<<<(h.fd.nx + 255) / 256, 256, 0, st>>>(d, out);
    return cudaGetLastError();
}

}  // namespace avl
