// avl_internal.cuh -- device-side data layout shared by the kernels and the
// host layer of the GB300 Vlasov-Hybrid library.
//
// HBM layout of one species (1d1v):
//   markers, double-buffered for re-sorting, structure of arrays:
//     FP32: cell int32[n], off f32[n] (position in cells = cell + off,
//           off in [0,1)), dv f32[n] (velocity relative to the reference
//           velocity of the marker's bin), f f32[n]
//     FP64: xi f64[n] (position in cells), dv f64[n], f f64[n]
//   bins: markers are grouped by velocity row block ("bin" = TV rows of the
//     velocity grid); bin_start[nbins+1] gives each bin's marker range.
//   grids are stored [v][x] (x fastest): f, n (= denominator of Eq. 4).
//   partial sums of each bin's window: [nbins][planes][W][nx].
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/avl.h"

namespace avl {

constexpr int MAXS = AVL_MAX_SPECIES;
constexpr int PD_THREADS = 256;     // push + deposit block
constexpr int PD_UNROLL = 4;        // markers in flight per thread
constexpr int FIN_THREADS = 256;    // finalize block
constexpr int FIN_XB = 16;          // x columns per finalize block
constexpr int FIELD_THREADS = 512;  // Poisson cluster block
constexpr int FIELD_CLUSTER = 8;    // CTAs in the Poisson cluster
constexpr int SORT_THREADS = 256;
constexpr long long WAIT_LIMIT = 1ll << 22;   // bounded mbarrier polls

// device-side error bits (Ctl::err)
enum : int { ERR_TIMEOUT = 1, ERR_NUMERIC = 2, ERR_CAPACITY = 4 };

struct SpDev {
    int nvdim, nx, nv[3], nvflat;
    int mobile;
    long long n;               // markers
    double q, m, qm;
    double vmin[3], dv[3], inv_dv[3];
    double dx;
    double qm_dt, dt_dx;       // (q/m) dt, dt/dx
    // binning by velocity row blocks (1d1v)
    int tv;                    // rows per bin
    int hw;                    // window rows beyond the bin on each side (CIC + drift halo)
    int hd;                    // rows a marker may wander out of its bin before a re-sort
    int W;                     // window rows = tv + 2 hw
    int nbins;
    int bin_base;              // first global bin index of this species
    // finalize blocks: FIN_XB x-columns times a group of rq velocity rows
    int nxb, rq, nrq, nfin, fin_base;
    // markers
    void* mx[2];               // FP32: int cell; FP64: double xi
    float* moff[2];            // FP32 only
    void* mv[2][3];            // velocity components (vx bin-relative)
    void* mf[2];
    int* bin_start[2];
    int* cursor;
    int* hist;
    // grids and scratch
    void* fgrid;               // [nvflat][nx] (storage precision)
    void* ngrid;
    void* partial;             // [nbins][planes][W][nx]
    double* ovf;               // [2][nvflat][nx] FP64 overflow num/den
    double* rho_part;          // [nrq][nx] charge of this species per row group
    double* dpart;             // [nfin][4] : N, Wkin, S, -
};

struct FieldDev {
    int nx, pow2, softening, ndiag;
    double L, dx, cP;
    double* rho;               // nx
    double* E64;               // nx
    float* E32;                // nx
    const double2* tw;         // exp(-2 pi i k / nx), k < nx
    const double* gmul;        // cP kappa / K^2 for m <= nx/2 (0 at m = 0 and Nyquist)
    double* diag;              // 3 + 3 ns
};

struct Ctl {
    int cur[MAXS];
    int sort_flag[MAXS];
    unsigned long long dirty[MAXS];
    unsigned long long ovf_count[MAXS];
    unsigned long long ovf_last[MAXS];
    unsigned long long nsort[MAXS];
    unsigned int scatter_done;
    int any_sort;
    long long step;
    int err;
};

struct StepArgs {
    int ns, prec, nvdim;
    int nbins_total, nfin_total;
    SpDev sp[MAXS];
    FieldDev fd;
    Ctl* ctl;
};

// kernel launchers (defined in the .cu files; all enqueue on `st`)
cudaError_t launch_pd1(const StepArgs& h, const StepArgs* d, int push, cudaStream_t st);
cudaError_t launch_fin1(const StepArgs& h, const StepArgs* d, int all_species, cudaStream_t st);
cudaError_t launch_field(const StepArgs& h, const StepArgs* d, int count_step,
                         unsigned long long sort_cond, cudaStream_t st);
cudaError_t launch_sort1(const StepArgs& h, const StepArgs* d, cudaStream_t st);
cudaError_t launch_init1(const StepArgs& h, const StepArgs* d, int s, const int lattice[4],
                         const avl_f0* f0_dev, unsigned long long seed, double jitter,
                         cudaStream_t st);
cudaError_t launch_set1(const StepArgs& h, const StepArgs* d, int s, long long n,
                        const double* x, const double* v, const double* f,
                        unsigned long long* bad, cudaStream_t st);
cudaError_t launch_get1(const StepArgs& h, const StepArgs* d, int s, double* x, double* v,
                        double* f, cudaStream_t st);
cudaError_t launch_getf(const StepArgs& h, int s, double* f, double* n, cudaStream_t st);

size_t pd1_smem_bytes(const SpDev& sp, int prec);
cudaError_t configure_vhs1(const StepArgs& h);
cudaError_t configure_field(const StepArgs& h);
// spectral tables of the Poisson solve (host) and the stand-alone solve
void spectral_tables(int nx, double L, double cP, int softening, double2* tw, double* gm);
size_t poisson_smem_bytes(int nx);
cudaError_t launch_poisson(const double* rho, double* E, int nx, const double2* tw, const double* gmul,
                           cudaStream_t st);

}  // namespace avl
