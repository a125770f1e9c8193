// avl_internal.cuh -- device-side data layout shared by the kernels and the
// host layer of the GB300 Vlasov-Hybrid library.
//
// HBM layout of one species (1d1v):
//   markers, double-buffered (a re-sorting step writes the markers sorted
//   by their keys into the other buffer before the push), structure of
//   arrays:
//     FP32: cell int32[n], off f32[n] (position in cells = cell + off, off in
//           [0,1)), dv f32[n], f f32[n]                      16 B per marker
//     FP64: X int64[n] (position: a count of 2^-52 cells), dv f64[n],
//           f f64[n]                                         24 B
//   Markers are sorted by their key, the lower velocity row of their
//   cloud-in-cell footprint (the "dual row", clamped to [0, nv)).  The marker
//   array is cut into chunks of M markers (chunk c = [c M, (c+1) M)); one CTA
//   owns one chunk.  dv is the velocity relative to the chunk's reference
//   row KB[c] (reference velocity vmin + KB[c] dv), so that FP32 keeps
//   velocity resolution at every |v|.
//   Grids are stored [v][x] (x fastest): f and n (denominator of Eq. 4).
//   Window partial sums of chunk c: [nchunk][planes][Wmax][nx] covering the
//   velocity rows [wrow0[c], wrow0[c] + Wmax).
//
// HBM layout of one species (1d3v):
//   markers as above plus v_y, v_z (FP32: cell, off, vx, vy, vz, f = 24 B);
//   velocities are absolute.  Sorted by pencil p = (jz + 1)(nvy + 1) + jy + 1
//   (jy, jz: dual rows of v_y, v_z, clamped to [-1, nv - 1]) and inside a
//   pencil by key k = jx + 1 (dual row of v_x, clamped likewise): seg[b][p][k]
//   is the first marker of key k of pencil p in buffer b, seg[b][p][nkey] the
//   end of the pencil.  Without a magnetic field v_y and v_z never change, so
//   a pencil's range is the same in both buffers; with one, every step re-sorts
//   the whole species by (pencil, key) into the other buffer.
//   Grids are stored [vz][vy][vx][x] (x fastest); acc[a] holds the numerator
//   and then the denominator of Eq. 4 for the deposit into accumulator a.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/avl.h"

namespace avl {

constexpr int MAXS = AVL_MAX_SPECIES;
constexpr int PD_THREADS = 512;     // push + deposit block
constexpr int MPT = 4;              // consecutive markers per thread and iteration
constexpr int CNT_THREADS = 512;    // key-count block
constexpr int HIST_S = 64;          // keys per chunk histogram
constexpr int HIST_R = 16;          // of which below the chunk's reference key
constexpr int HALO = 2;             // window rows beyond the chunk's keys (one step of drift)
constexpr int WIN_SPARE = 4;        // further window rows for the key spread between re-sorts
constexpr int FIN_THREADS = 256;    // finalize block
constexpr int FIN_XB = 16;          // x columns per finalize block
constexpr int FIELD_THREADS = 512;  // Poisson cluster block
constexpr int FIELD_CLUSTER = 8;    // CTAs in the Poisson cluster
// table of the FP64 entropy logarithm (log_tab): one entry per 1/2048 of the
// mantissa interval [1, 2)
constexpr int LOG_TAB_BITS = 11;
constexpr int LOG_TAB_N = 1 << LOG_TAB_BITS;
constexpr long long WAIT_LIMIT = 1ll << 22;   // bounded mbarrier polls: the default limit of a first wait
                                              // (Ctl::wait_limit) and the limit of the drain that follows
                                              // a first wait that gave up
constexpr int P3_THREADS = 256;     // 1d3v pencil block (one thread per x column and CPT3 columns)
constexpr int FIN3_X = 32;          // 1d3v finalize: x columns per block
constexpr int FIN3_R = 8;           //                row lanes per block
constexpr int NV3_MAX = 1024;       // 1d3v: largest nv[0] (key histogram of a pencil in shared memory)
constexpr int GREEN_MAX = 1024;     // largest nx solved by the circulant product (adjoint engine)

// elements of one deposit-window plane (numerator, denominator or reference)
// of a 1d1v chunk: Wmax rows x nx columns, padded to a multiple of 4 so that
// every plane (FP32 or FP64) starts and ends on a 16-byte boundary, as the
// bulk copies of the window need
__host__ __device__ inline int win_plane(int W, int nx) { return (W * nx + 3) & ~3; }

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
    // chunks
    int M;                     // markers per chunk (multiple of 64)
    int nchunk;                // chunks (0: no markers)
    int chunk_base;            // first global chunk index of this species
    int Wmax;                  // window rows
    unsigned div_m;            // magic multiplier and shift for slot / M
    int div_l;
    // markers
    void* mx[2];               // FP32: int cell; FP64: int64 X (2^-52 cells)
    float* moff[2];            // FP32 only
    void* mv[2][3];            // velocity components (vx chunk-relative)
    void* mf[2];
    void* mwq[2];              // FP64 1d3v: [n][4] weights of the marker's four (v_y, v_z) cells (the
                               // pencil's planes; 0 when the footprint misses the grid), per buffer
    int* KB[2];                // [nchunk] reference key of each chunk, per buffer
    // re-sort tables; cnt / far_cnt are double-buffered: [hsel] holds the key
    // counts of the current state, [1 - hsel] collects those of the next
    int* cnt[2];               // [nchunk][HIST_S] key histogram of each chunk
    int* far_cnt[2];           // [nv] markers whose key is outside their chunk's histogram
    int* offs;                 // [nchunk][HIST_S] first slot in the re-sorted layout
    int* far_cur;              // [nv] slot cursors of the far markers
    int* base_new;             // [nv + 1] first slot of each key in the re-sorted layout
    int* wrow0;                // [nchunk] first deposit-window row of each chunk
    int* shift[2];             // [nx] velocity rows the field moves a marker at x in one step
                               // (rounded): [shsel] for this step's field, the other for the
                               // previous step's.  Deposit windows and their partial sums are
                               // stored shifted back by it, column by column
    int* kref_tmp;             // [nchunk] scratch of the marker creation path
    // grids and scratch
    void* fgrid;               // [nvflat][nx] (storage precision)
    void* ngrid;
    void* partial;             // [nchunk][planes][Wmax][nx]
    double* ovf;               // [2][nvflat][nx] FP64 overflow num/den
    int* ovf_tag;              // [nvflat] step tag (step + 1) of the last overflow into each row
    double* rho_part;          // [nrq][nx] charge of this species per row group
    double* dpart;             // [nfin][4] : N, Wkin, S, -
    // finalize blocks: FIN_XB x-columns times a group of rq velocity rows
    int nxb, rq, nrq, nfin, fin_base;
    // 1d3v
    int npen;                  // (nv[1] + 1) (nv[2] + 1) pencils
    int nkey;                  // nv[0] + 1 keys per pencil
    int pen_base;              // first global pencil block of this species
    int* seg[2];               // [npen][nkey + 1] first marker of every key, per buffer
    void* acc[2];              // [2][nvflat][nx] numerator, denominator of the deposit
    void* v2row;               // [nvflat] |v|^2 at the centre of every velocity cell
    int* kcount;               // [npen * nkey] bucket counts (zero between operations)
    int* kcur;                 // [npen * nkey] slot cursors of a creation or global re-sort
    int* ktile;                // [ceil(npen * nkey / 1024)] bucket counts per scan tile
};

struct FieldDev {
    int nx, pow2, softening, ndiag;
    int resort_drift;          // 1d1v: re-sort whenever the field drifts markers a row or more (default
                               // off: the per-column shift tables already move the windows with the drift)
    int resort_miss;           // 1d1v: re-sort when more than n / resort_miss markers miss their window
                               // (default 30: the overflow path takes up to ~3 % cheaper than a re-sort)
    double L, dx, cP;
    double we_scale;           // dx / (2 cP): field energy per sum of E^2 over the cells
    double* rho;               // nx
    double* E64;               // nx
    float* E32;                // nx
    const double2* tw;         // exp(-2 pi i k / nx), k < nx
    const double* gmul;        // cP kappa / K^2 for m <= nx/2 (0 at m = 0 and Nyquist)
    const double* green;       // nx <= GREEN_MAX: G of E = G (circulant) rho, else null
    double* diag;              // 3 + 3 ns
    const double2* logtab;     // [LOG_TAB_N] (log c_j, 1 / c_j) of the FP64 entropy logarithm (log_tab)
    double* hist;              // field history for marker refinement: [hist_cap][nx] FP64, or null;
                               // slot k holds E of the state after step hist_origin + k
    int hist_cap;
    long long hist_origin;
    double B[3];               // 1d3v: static background magnetic field (Boris push)
    int magnetized;            // B != 0 (1d3v): push, global re-sort, deposit
};

struct Ctl {
    int cur[MAXS];             // buffer holding the current markers
    int sort_now[MAXS];        // this step re-sorts the markers before the push
    int sort_next[MAXS];       // decided by the field kernel for the next step
    int hsel[MAXS];            // which cnt / far_cnt buffer holds the current counts
    unsigned long long ovf_count[MAXS];
    unsigned long long ovf_last[MAXS];
    unsigned long long nsort[MAXS];
    unsigned long long uncovered[MAXS];   // markers outside their chunk's best window (decision input)
    int shift_min[MAXS][2], shift_max[MAXS][2];   // range of each shift table
    int shsel[MAXS];           // which shift table belongs to this step's field
    long long step;
    int err;
    long long wait_limit;      // polls of the first bounded wait on a bulk copy (avl_set_wait_limit)
    // 1d3v
    int asel[MAXS];                        // accumulator the next deposit writes into
    unsigned long long movers[MAXS];       // markers whose key left their segment (this pass)
    unsigned long long far_movers[MAXS];   // of which two or more rows away
    unsigned long long movers_last[MAXS];
};

struct StepArgs {
    int ns, prec, nvdim;
    int nchunk_total, nfin_total;
    int npen_total;
    SpDev sp[MAXS];
    FieldDev fd;
    Ctl* ctl;
};

// Several independent runs advanced by one launch per kernel class: block g
// of a batched launch belongs to run r with base[r] <= g < base[r + 1] (its
// local block g - base[r]); the field kernel's cluster c belongs to run c.
struct BatchMap {
    int nrun;
    const StepArgs* const* args;   // [nrun] each run's arguments (device)
    const int* pd_base;            // [nrun + 1] push + deposit blocks
    const int* fin_base;           // [nrun + 1] finalize blocks
};

// run and local block of this block (A itself and blockIdx.x when bm is null)
__device__ __forceinline__ const StepArgs* batch_run(const StepArgs* A, const BatchMap* bm, const int* base, int& g)
{
    g = (int)blockIdx.x;
    if (!bm) return A;
    int lo = 0, hi = bm->nrun;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (base[mid] <= g) lo = mid; else hi = mid;
    }
    g -= base[lo];
    return bm->args[lo];
}

// kernel launchers (defined in the .cu files; all enqueue on `st`).
// launch_count1: key histograms of the current markers (after creation).
// launch_rs1: markers of the species the field kernel marked into the layout
//             sorted by their current keys (other buffer; a no-op otherwise).
// launch_pd1 mode: 0 = refresh (every species with markers: deposit only)
//                  1 = step (mobile species: push, deposit, write back in
//                      place, key histograms of the new state)
cudaError_t launch_count1(const StepArgs& h, const StepArgs* d, cudaStream_t st);
cudaError_t launch_rs1(const StepArgs& h, const StepArgs* d, cudaStream_t st);
cudaError_t launch_pd1(const StepArgs& h, const StepArgs* d, int mode, cudaStream_t st);
cudaError_t launch_fin1(const StepArgs& h, const StepArgs* d, int all_species, cudaStream_t st);
cudaError_t launch_field(const StepArgs& h, const StepArgs* d, int count_step, cudaStream_t st);
// batched forms (bm on the device; blocks = totals over the runs, smem = the
// largest of the runs' needs, set beforehand by configure_batch1)
cudaError_t launch_rs1_batch(int prec, const BatchMap* bm, int blocks, cudaStream_t st);
cudaError_t launch_pd1_batch(int prec, const BatchMap* bm, int blocks, int smem, int mode, cudaStream_t st);
cudaError_t launch_fin1_batch(int prec, const BatchMap* bm, int blocks, int all_species, cudaStream_t st);
cudaError_t launch_field_batch(const BatchMap* bm, int nrun, int smem, int count_step, cudaStream_t st);
cudaError_t configure_batch1(int prec, int pd_smem, int field_smem);
size_t field_smem_bytes(const StepArgs& h);
int pd1_smem_needed(const StepArgs& h);
// markers from the lattice generator or from caller arrays into the sorted
// layout of buffer 0 of species s
cudaError_t launch_init1(const StepArgs& h, const StepArgs* d, int s, const int lattice[4],
                         const avl_f0* f0_dev, unsigned long long seed, double jitter,
                         cudaStream_t st);
cudaError_t launch_set1(const StepArgs& h, const StepArgs* d, int s, long long n,
                        const double* x, const double* v, const double* f,
                        unsigned long long* bad, cudaStream_t st);
cudaError_t launch_get1(const StepArgs& h, const StepArgs* d, int s, double* x, double* v,
                        double* f, cudaStream_t st);
cudaError_t launch_getf(const StepArgs& h, int s, double* f, double* n, cudaStream_t st);
// marker refinement (1d1v): count new markers on a jittered lattice of the box
// of cells at the current time, traced back nhist steps through Ehist (E of
// the species' initial state first) to f = f0 at the foot; FP64 outputs
cudaError_t launch_refine1(const StepArgs& h, int s, const int box[4], const int lattice[2], const avl_f0* f0_dev,
                           unsigned long long seed, double jitter, double dt, int nhist, const double* Ehist,
                           long long count, double* x, double* v, double* f, cudaStream_t st);

// 1d3v (k_vhs3.cu).  launch_pd3 mode as launch_pd1, and 2 = deposit only,
// mobile species (after a magnetized push and re-sort); launch_sort3 re-sorts
// the pencils of the species the field kernel marked (a no-op otherwise).
// launch_bpush3: Boris push of species s in place, counting the new buckets;
// launch_rsort3: the counted markers of species s re-sorted by (pencil, key)
// into the other buffer, which becomes current.
cudaError_t configure_vhs3(const StepArgs& h);
cudaError_t launch_pd3(const StepArgs& h, const StepArgs* d, int mode, cudaStream_t st);
cudaError_t launch_fin3(const StepArgs& h, const StepArgs* d, int all_species, cudaStream_t st);
cudaError_t launch_sort3(const StepArgs& h, const StepArgs* d, cudaStream_t st);
cudaError_t launch_bpush3(const StepArgs& h, const StepArgs* d, int s, cudaStream_t st);
cudaError_t launch_rsort3(const StepArgs& h, const StepArgs* d, int s, cudaStream_t st);
cudaError_t launch_init3(const StepArgs& h, const StepArgs* d, int s, const int lattice[4],
                         const avl_f0* f0_dev, unsigned long long seed, double jitter,
                         cudaStream_t st);
cudaError_t launch_set3(const StepArgs& h, const StepArgs* d, int s, long long n,
                        const double* x, const double* v, const double* f,
                        unsigned long long* bad, cudaStream_t st);
cudaError_t launch_get3(const StepArgs& h, const StepArgs* d, int s, double* x, double* v,
                        double* f, cudaStream_t st);
// f (and n) of the current deposit in the caller's [x][vx][vy][vz] order;
// asel = accumulator selector after the last deposit
cudaError_t launch_getf3(const StepArgs& h, int s, int asel, double* f, double* n, cudaStream_t st);
size_t pd3_smem_bytes(int nx, int nkey, int prec);

// output moments of species s ([2 + nvdim][nx], device, FP64) and the field
// residual ([nx]) of the current state (k_moments.cu)
cudaError_t launch_moments(const StepArgs& h, const StepArgs* d, int s, double* out, cudaStream_t st);
cudaError_t launch_residual(const StepArgs& h, const StepArgs* d, double* out, cudaStream_t st);

// discrete adjoint of the 1d1v step (k_adjoint.cu): the species' lattice
// parameters of their last creation, theta = the f0 of species theta_s
struct AdjSpec {
    int theta_s, nsteps, ckpt_every;
    long long n[MAXS];
    int lat[MAXS][2];
    unsigned long long seed[MAXS];
    double jitter[MAXS];
    avl_f0 f0[MAXS];
};
struct AdjEngine;   // buffers, kept by the context between calls
cudaError_t adjoint_run(AdjEngine** eng, const StepArgs& h, const StepArgs* d, const AdjSpec& spec,
                        cudaStream_t st, double* dJ_amp, double* dJ_u, double* J);
void adjoint_free(AdjEngine* e);

size_t pd1_smem_bytes(const SpDev& sp, int prec);
size_t window_bytes(const SpDev& sp, int prec);
cudaError_t configure_vhs1(const StepArgs& h);
cudaError_t configure_field(const StepArgs& h);
cudaError_t configure_field_bytes(int bytes);
// spectral tables of the Poisson solve (host) and the stand-alone solve
void spectral_tables(int nx, double L, double cP, int softening, double2* tw, double* gm);
size_t poisson_smem_bytes(int nx);
void green_table(int nx, const double* gm, double* G);
cudaError_t launch_poisson_dense(const double* rho, double* E, int nx, const double* G, cudaStream_t st);
cudaError_t launch_poisson(const double* rho, double* E, int nx, const double2* tw, const double* gmul,
                           cudaStream_t st);
// table of the FP64 entropy logarithm: tab[j] = (log c_j, 1 / c_j), c_j = 1 + (j + 1/2) / 128
cudaError_t init_log_table(double2* tab, cudaStream_t st);

}  // namespace avl
