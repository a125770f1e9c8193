// k_field.cu -- net charge density and spectral Poisson solve (Sec. 3.1,
// Eq. 5 / Eq. 6a-c), diagnostics row (Sec. 3.4.1) and the re-sort decision.
//
// One thread-block cluster of FIELD_CLUSTER CTAs.  Every CTA sums the charge
// partials of a slice of x over all species and velocity row blocks and
// writes its slice into CTA 0's shared memory (distributed shared memory);
// CTA 0 then runs an FP64 real FFT of length nx (a complex radix-2 FFT of
// length nx/2 with the even/odd split), multiplies by -i cP kappa / K^2,
// transforms back, and writes E in FP64 and FP32.  A direct DFT serves grid
// sizes that are not a power of two.  Beside the solve, CTAs 1 .. decide the
// next step's 1d1v re-sorts and prepare their slots, and the last CTA sums
// the diagnostics.
#include <cooperative_groups.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "avl_internal.cuh"
#include "common.cuh"
#include "resort.cuh"

namespace cg = cooperative_groups;

namespace avl {

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 conj2(double2 a) { return make_double2(a.x, -a.y); }

// in-place radix-2 decimation-in-time FFT of length M (a power of two) on
// shared memory, input already in bit-reversed order; tw[k] = exp(-2 pi i
// k / N) for k = 0 .. M with N = 2 M (the copy staged in shared memory, or
// the global table for large grids); the inverse uses the conjugate
// twiddles (no scaling).  One butterfly per thread and
// stage: an FP64 warp instruction occupies its SM sub-partition for the same
// time whatever the number of active lanes, so the butterflies are packed
// into full warps.  The first two stages, whose twiddles are 1 and -i (+i
// for the inverse), take no multiplies.
__device__ void fft_pow2(double2* a, int M, const double2* tw, bool inverse)
{
    // stage 1: (2 t, 2 t + 1), w = 1
    for (int t = threadIdx.x; t < M / 2; t += blockDim.x) {
        const double2 u = a[2 * t], v = a[2 * t + 1];
        a[2 * t] = cadd(u, v);
        a[2 * t + 1] = csub(u, v);
    }
    __syncthreads();
    if (M >= 4) {
        // stage 2: (4 g + k, 4 g + k + 2), w = 1 for k = 0 and -i (+i) for k = 1
        for (int t = threadIdx.x; t < M / 2; t += blockDim.x) {
            const int i1 = 4 * (t >> 1) + (t & 1), i2 = i1 + 2;
            const double2 u = a[i1], x = a[i2];
            const double2 v = (t & 1) ? (inverse ? make_double2(-x.y, x.x) : make_double2(x.y, -x.x)) : x;
            a[i1] = cadd(u, v);
            a[i2] = csub(u, v);
        }
        __syncthreads();
    }
    for (int len = 8; len <= M; len <<= 1) {
        const int half = len >> 1;
        const int step = 2 * M / len;
        for (int t = threadIdx.x; t < M / 2; t += blockDim.x) {
            const int grp = t / half, k = t - grp * half;
            const int i1 = grp * len + k, i2 = i1 + half;
            double2 w = tw[k * step];
            if (inverse) w.y = -w.y;
            const double2 u = a[i1];
            const double2 v = cmul(a[i2], w);
            a[i1] = cadd(u, v);
            a[i2] = csub(u, v);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ int bitrev(int x, int bits) { return (int)(__brev((unsigned)x) >> (32 - bits)); }

// Shared memory of the solve: rho / E (nx doubles), the spectrum (nx/2 + 2
// complex) and, for power-of-two nx up to POISSON_STAGE_MAX, the staged
// tables: twiddles (nx/2 + 1 complex) and multipliers (nx/2 + 1 doubles);
// larger grids read the tables from global memory.
constexpr int POISSON_STAGE_MAX = 4096;
__host__ __device__ inline size_t poisson_rho_bytes(int nx) { return ((size_t)nx * 8 + 15) / 16 * 16; }
__host__ __device__ inline size_t poisson_work_bytes(int nx) { return ((size_t)nx / 2 + 2) * 16; }
__host__ __device__ inline bool poisson_pow2(int nx) { return nx >= 4 && (nx & (nx - 1)) == 0; }
__host__ __device__ inline bool poisson_stage(int nx) { return poisson_pow2(nx) && nx <= POISSON_STAGE_MAX; }
__host__ __device__ inline size_t poisson_smem_bytes_dev(int nx)
{
    return poisson_rho_bytes(nx) + poisson_work_bytes(nx) + (poisson_stage(nx) ? ((size_t)nx / 2 + 1) * 24 : 0);
}

// 1 / (4 M) for M = nx/2 = 2^bits: the halvings of the even/odd split and
// the 1/M of the inverse transform, an exact power of two set from its
// exponent (no FP64 division)
__device__ __forceinline__ double poisson_scale(int bits)
{
    return __longlong_as_double((long long)(1023 - bits - 2) << 52);
}

__device__ __forceinline__ int log2_pow2(int M)
{
    int bits = 0;
    while ((1 << bits) < M) ++bits;
    return bits;
}

// Tables of the power-of-two solve into shared memory: twiddles
// exp(-2 pi i k / nx) and multipliers gmul[k] / (4 M), k = 0 .. nx/2.  Whole
// block; the caller synchronises before poisson_spectral.
__device__ void stage_tables(double2* tw_s, double* gm_s, const double2* __restrict__ tw,
                             const double* __restrict__ gmul, int nx)
{
    const double c = poisson_scale(log2_pow2(nx / 2));
    for (int k = threadIdx.x; k <= nx / 2; k += blockDim.x) {
        tw_s[k] = tw[k];
        gm_s[k] = gmul[k] * c;
    }
}

// Spectral Poisson solve (Eq. 5 / Eq. 6a-c) by the whole block: rho_s holds
// rho in shared memory (nx doubles) and holds E on return; work is shared
// scratch of nx/2 + 2 complex values; tw_s the twiddles for the power-of-two
// path (staged in shared memory or the global table), gm_s the staged
// multipliers (already scaled; null: gmul scaled here)
// (power-of-two nx); tw[k] = exp(-2 pi i k / nx) and gmul[m] = cP kappa_m /
// K2_m (zero at m = 0 and at the Nyquist mode) in global memory.
//
// Power-of-two nx: rho packed as z_n = rho_2n + i rho_2n+1 goes through one
// complex FFT of length M = nx/2; the modes m and M - m are unpacked
// together (X = rho-hat, Eq. 6a), multiplied by -i g (Eq. 6b-c) and packed
// back for the inverse transform, whose output pairs are E_2n, E_2n+1.  The
// halvings of the even/odd split and the 1/M of the inverse, all powers of
// two, are folded into g.
__device__ void poisson_spectral(double* rho_s, double2* work, const double2* tw_s, const double* gm_s, int nx,
                                 int pow2, const double2* __restrict__ tw, const double* __restrict__ gmul)
{
    if (pow2) {
        const int M = nx / 2;
        const int bits = log2_pow2(M);
        for (int n = threadIdx.x; n < M; n += blockDim.x)
            work[bitrev(n, bits)] = make_double2(rho_s[2 * n], rho_s[2 * n + 1]);
        __syncthreads();
        fft_pow2(work, M, tw_s, false);
        double2* Y = reinterpret_cast<double2*>(rho_s);   // M complex values over the nx doubles
        // thread t takes the modes m = t and M - t; thread 0 takes m = M/2,
        // its own partner, and Y_0 = 0 (g vanishes at m = 0 and at the
        // Nyquist mode M), so that M/2 threads fill whole warps
        if (threadIdx.x == 0) Y[0] = make_double2(0.0, 0.0);
        for (int t = threadIdx.x; t < M / 2; t += blockDim.x) {
            const int m = t == 0 ? M / 2 : t;
            const int p = M - m;
            const double2 A = work[m];
            const double2 B = conj2(work[p]);
            const double2 S = cadd(A, B), D = csub(A, B);
            // W^p = -conj(W^m), so with V = W^m (-i D):
            // 2 X_m = S + V,  2 X_p = conj(S) + W^p (i conj D) = conj(S - V)
            const double2 twm = tw_s[m];
            const double2 V = cmul(twm, make_double2(D.y, -D.x));
            const double2 Xm = cadd(S, V), Xp = conj2(csub(S, V));
            // E-hat = -i g X, with the scale folded into g
            const double c = gm_s ? 1.0 : poisson_scale(bits);
            const double gm = gm_s ? gm_s[m] : gmul[m] * c, gp = gm_s ? gm_s[p] : gmul[p] * c;
            const double2 Em = make_double2(gm * Xm.y, -gm * Xm.x);
            const double2 Ep = make_double2(gp * Xp.y, -gp * Xp.x);
            // Y_m = F + i O with F = E_m + conj E_p, O = (E_m - conj E_p) conj(W^m);
            // for the partner F' = conj(F) and O' = conj(O)
            const double2 F = cadd(Em, conj2(Ep)), O = cmul(csub(Em, conj2(Ep)), conj2(twm));
            Y[bitrev(m, bits)] = make_double2(F.x - O.y, F.y + O.x);
            if (p != m) Y[bitrev(p, bits)] = make_double2(F.x + O.y, -F.y + O.x);
        }
        __syncthreads();
        fft_pow2(Y, M, tw_s, true);
    } else {
        // direct DFT: Ehat_m for m = 1 .. (nx-1)/2, then E_i = (2/N) sum Re(Ehat_m e^{+i})
        const int mmax = (nx - 1) / 2;
        for (int m = 1 + threadIdx.x; m <= mmax; m += blockDim.x) {
            double rr = 0.0, ri = 0.0;
            for (int i = 0; i < nx; ++i) {
                const double2 w = tw[(int)(((long long)m * i) % nx)];
                rr += rho_s[i] * w.x;
                ri += rho_s[i] * w.y;
            }
            const double g = gmul[m];
            work[m] = make_double2(g * ri, -g * rr);   // -i g (rr + i ri)
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            double acc = 0.0;
            for (int m = 1; m <= mmax; ++m) {
                const double2 w = tw[(int)(((long long)m * i) % nx)];
                // Re(E_m * conj(w))
                acc += work[m].x * w.x + work[m].y * w.y;
            }
            rho_s[i] = 2.0 * acc / (double)nx;
        }
        __syncthreads();
    }
}

// Markers a chunk's best deposit window holds: the largest sum of wk
// consecutive bins of its HIST_S-bin key histogram (the window best_window
// places).  Called by a whole warp with lane l holding bins 2 l and 2 l + 1
// (one coalesced load); a warp scan.
__device__ __forceinline__ int best_cover_warp(int2 h, int wk)
{
    static_assert(HIST_S == 64, "two bins per lane");
    const int lane = threadIdx.x & 31;
    int S = h.x + h.y;   // inclusive prefix of the bin pairs over the lanes
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, S, o);
        if (lane >= o) S += y;
    }
    // P(i) = sum of bins [0, i): P(2 l + 2) = S(l), P(2 l + 1) = S(l) - h.y(l)
    auto P = [&](int i) {
        const int src = max(i - 1, 0) >> 1;
        const int Ss = __shfl_sync(0xffffffffu, S, src);
        const int hy = __shfl_sync(0xffffffffu, h.y, src);
        return i == 0 ? 0 : ((i & 1) ? Ss - hy : Ss);
    };
    int best = 0;
    for (int q = 0; q < 2; ++q) {
        const int r = 2 * lane + q;
        const int a = P(r), b = P(min(r + wk, HIST_S));
        if (r + wk <= HIST_S) best = max(best, b - a);
    }
    return __reduce_max_sync(0xffffffffu, best);
}

constexpr int FIELD_DECIDE = FIELD_CLUSTER - 2;   // CTAs 1 .. FIELD_DECIDE decide the re-sorts
constexpr int FIELD_DIAG = FIELD_CLUSTER - 1;     // the last CTA sums the diagnostics

// After a step: CTA 1 + (s mod FIELD_DECIDE) of the field cluster decides,
// for mobile species s, whether the next step re-sorts its markers before
// the push (when the field drifts markers a row or more, or the best deposit
// windows of the chunks, placed from the key counts of the new state, would
// miss more than a small fraction of the markers) and if so prepares the
// slots and the key histograms of the re-sorted chunks; then CTAs 1.. clear
// the key counts consumed by this step for reuse.
__device__ __forceinline__ unsigned dynamic_smem_bytes()
{
    unsigned r;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}

__device__ void resort_work(const StepArgs* __restrict__ A, int rank, int* dyn)
{
    const size_t dyn_bytes = dynamic_smem_bytes();
    const Ctl* ctl = A->ctl;
    __shared__ unsigned long long miss;
    for (int s = rank - 1; rank <= FIELD_DECIDE && s < A->ns; s += FIELD_DECIDE) {
        const SpDev& sp = A->sp[s];
        const int hs = ctl->hsel[s];
        if (!sp.mobile || sp.nchunk == 0) continue;
        const int cur_after = ctl->sort_now[s] ? 1 - ctl->cur[s] : ctl->cur[s];
        const int* kref = sp.KB[cur_after];
        const int* cnt = sp.cnt[1 - hs];
        const int* far = sp.far_cnt[1 - hs];
        // the scan of the re-sort in this CTA's dynamic shared memory (unused
        // by the CTAs other than 0) when the key range fits
        int* base_s = ((size_t)sp.nvflat + 1) * 4 <= dyn_bytes ? dyn : nullptr;
        // markers outside the best window of their chunk (a warp per chunk)
        if (threadIdx.x == 0) miss = 0;
        __syncthreads();
        const int wk = max(1, min(HIST_S, sp.Wmax - 2 * HALO - 1));
        unsigned long long my = 0;
        // two chunks per warp and pass, the next pass's histograms loaded ahead
        const int nw = FIELD_THREADS / 32, lane = threadIdx.x & 31;
        const int2* cnt2 = reinterpret_cast<const int2*>(cnt);
        auto load = [&](int c) { return c < sp.nchunk ? cnt2[(size_t)c * (HIST_S / 2) + lane] : make_int2(0, 0); };
        int c = threadIdx.x >> 5;
        int2 ha = load(c), hb = load(c + nw);
        for (; c < sp.nchunk; c += 2 * nw) {
            const int2 a = ha, b = hb;
            ha = load(c + 2 * nw);
            hb = load(c + 3 * nw);
            const int cov_a = best_cover_warp(a, wk), cov_b = best_cover_warp(b, wk);
            if (lane == 0) {
                const long long beg = (long long)c * sp.M;
                my += (unsigned long long)(min(beg + sp.M, sp.n) - beg - cov_a);
                if (c + nw < sp.nchunk) {
                    const long long beg_b = (long long)(c + nw) * sp.M;
                    my += (unsigned long long)(min(beg_b + sp.M, sp.n) - beg_b - cov_b);
                }
            }
        }
        if (my) atomicAdd(&miss, my);
        __syncthreads();
        // rows this step's field drifts markers (its table is not the one
        // CTA 0 is rewriting now); at a row or more, re-sort every step
        const int ssel = ctl->shsel[s];
        const int drift = max(abs(ctl->shift_min[s][ssel]), abs(ctl->shift_max[s][ssel]));
        const bool resort = (A->fd.resort_drift && drift >= 1) ||
                            miss * (unsigned long long)A->fd.resort_miss > (unsigned long long)sp.n;
        if (threadIdx.x == 0) {
            Ctl* cw = A->ctl;
            cw->uncovered[s] = miss;
            cw->sort_next[s] = resort ? 1 : 0;
        }
        if (resort) {
            scan_layout(sp, kref, cnt, far, true, sp.KB[1 - cur_after], base_s);
            // the next step deposits from the re-sorted layout: its window
            // placement takes the key histograms of the re-sorted chunks
            sorted_chunk_hist(sp, sp.KB[1 - cur_after], sp.cnt[1 - hs], base_s ? base_s : sp.base_new);
        }
        __syncthreads();
    }
    // clear cnt[hs] and far_cnt[hs] of every species for the next step's counting
    const int nclr = FIELD_CLUSTER - 1;
    const int r = rank - 1;
    for (int s = 0; s < A->ns; ++s) {
        const SpDev& sp = A->sp[s];
        if (!sp.mobile || sp.nchunk == 0) continue;
        const int hs = ctl->hsel[s];
        const size_t ncnt = (size_t)sp.nchunk * HIST_S;
        for (size_t i = (size_t)r * blockDim.x + threadIdx.x; i < ncnt; i += (size_t)nclr * blockDim.x)
            sp.cnt[hs][i] = 0;
        for (int i = r * blockDim.x + threadIdx.x; i < sp.nvflat; i += nclr * blockDim.x) sp.far_cnt[hs][i] = 0;
    }
}

// per-species sums of the finalize blocks' diagnostics (N, W_kin, S; fixed
// order per thread, then over the warps) into out[3 s + q] (CTA 0's shared
// memory); called by the whole block of CTA FIELD_DIAG
__device__ void diag_sums(const StepArgs* __restrict__ A, double* out)
{
    __shared__ double dsum[3 * MAXS][FIELD_THREADS / 32];
    const int ns = A->ns;
    for (int s = 0; s < ns; ++s) {
        const SpDev& sp = A->sp[s];
        double N = 0.0, Wk = 0.0, S = 0.0;
        for (int k = threadIdx.x; k < sp.nfin; k += FIELD_THREADS) {
            N += sp.dpart[(size_t)k * 4 + 0];
            Wk += sp.dpart[(size_t)k * 4 + 1];
            S += sp.dpart[(size_t)k * 4 + 2];
        }
        for (int o = 16; o > 0; o >>= 1) {
            N += __shfl_down_sync(0xffffffffu, N, o);
            Wk += __shfl_down_sync(0xffffffffu, Wk, o);
            S += __shfl_down_sync(0xffffffffu, S, o);
        }
        if ((threadIdx.x & 31) == 0) {
            dsum[3 * s + 0][threadIdx.x >> 5] = N;
            dsum[3 * s + 1][threadIdx.x >> 5] = Wk;
            dsum[3 * s + 2][threadIdx.x >> 5] = S;
        }
    }
    __syncthreads();
    if (threadIdx.x < 3 * ns) {
        double v = 0.0;
        for (int w = 0; w < FIELD_THREADS / 32; ++w) v += dsum[threadIdx.x][w];
        out[threadIdx.x] = v;
    }
}

__global__ void __cluster_dims__(FIELD_CLUSTER, 1, 1) __launch_bounds__(FIELD_THREADS)
    k_field(const StepArgs* __restrict__ A0, int count_step, const BatchMap* __restrict__ bm)
{
    // one cluster per run in a batched launch
    const StepArgs* __restrict__ A = bm ? bm->args[blockIdx.x / FIELD_CLUSTER] : A0;
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const FieldDev& fd = A->fd;
    const int nx = fd.nx;
    double* rho_s = reinterpret_cast<double*>(smem);                                  // nx
    double2* work = reinterpret_cast<double2*>(smem + poisson_rho_bytes(nx));          // nx/2 + 2
    double2* tw_s = reinterpret_cast<double2*>(smem + poisson_rho_bytes(nx) + poisson_work_bytes(nx));
    double* gm_s = reinterpret_cast<double*>(tw_s + nx / 2 + 1);
    __shared__ double red[FIELD_THREADS / 32];
    __shared__ double dfin[3 * MAXS];   // per-species diagnostics sums (written by CTA FIELD_DIAG)
    __shared__ float shf_s[MAXS];       // per species: rows per unit field and step (shift table)
    __shared__ int tgt_s[MAXS];         // per species: shift table this kernel writes

    // CTA 0 stages the tables of the solve while the cluster sums rho
    const bool staged = poisson_stage(nx);
    if (rank == 0 && staged) stage_tables(tw_s, gm_s, fd.tw, fd.gmul, nx);

    // --- rho slice: sum over species and row blocks (fixed order) --------
    // tpx threads per column (a power of two up to 32) take every tpx-th
    // partial row and are summed by a fixed shuffle tree
    double* rho0 = cluster.map_shared_rank(rho_s, 0);
    const int per = (nx + FIELD_CLUSTER - 1) / FIELD_CLUSTER;
    const int xlo = rank * per, xhi = min(nx, xlo + per);
    {
        int tpx = 1;
        while (tpx < 32 && tpx * 2 * max(per, 1) <= FIELD_THREADS) tpx *= 2;
        const int part = threadIdx.x & (tpx - 1);
        const int cols = FIELD_THREADS / tpx;
        int nrows = 0;
        for (int s = 0; s < A->ns; ++s) nrows += A->sp[s].nrq;
        for (int x0 = xlo; x0 < xhi; x0 += cols) {
            const int x = x0 + threadIdx.x / tpx;
            double r = 0.0;
            if (x < xhi) {
                int s = 0, base = 0;
                for (int k = part; k < nrows; k += tpx) {
                    while (k - base >= A->sp[s].nrq) base += A->sp[s++].nrq;
                    r += A->sp[s].rho_part[(size_t)(k - base) * nx + x];
                }
            }
            for (int o = tpx >> 1; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o, tpx);
            if (part == 0 && x < xhi) rho0[x] = r;
        }
    }
    cluster.sync();
    if (rank != 0) {
        if (rank == FIELD_DIAG) diag_sums(A, cluster.map_shared_rank(dfin, 0));
        if (count_step) resort_work(A, rank, reinterpret_cast<int*>(smem));
        cluster.sync();
        return;
    }

    // --- CTA 0: Poisson --------------------------------------------------
    for (int x = threadIdx.x; x < nx; x += FIELD_THREADS) fd.rho[x] = rho_s[x];
    // per-species constants of the shift tables: loads issued before the
    // solve, their values used after it
    double qm_dt = 0.0, inv_dv = 0.0;
    int mobile = 0, shsel = 0;
    if (threadIdx.x < A->ns) {
        const SpDev& sp = A->sp[threadIdx.x];
        mobile = sp.mobile;
        qm_dt = sp.qm_dt;
        inv_dv = sp.inv_dv[0];
        shsel = A->ctl->shsel[threadIdx.x];
    }
    poisson_spectral(rho_s, work, staged ? tw_s : fd.tw, staged ? gm_s : nullptr, nx, fd.pow2, fd.tw, fd.gmul);
    if (threadIdx.x < A->ns) {
        shf_s[threadIdx.x] = mobile ? (float)(qm_dt * inv_dv) : 0.f;
        tgt_s[threadIdx.x] = count_step ? 1 - shsel : shsel;
    }
    const double* E_s = rho_s;   // E, FP64, in shared memory
    // --- E in FP64 and FP32, field energy, diagnostics row -----------------
    float* E32_s = reinterpret_cast<float*>(work);   // the spectrum is no longer needed
    for (int x = threadIdx.x; x < nx; x += FIELD_THREADS) {
        const double e = E_s[x];
        const float e32 = (float)e;
        fd.E64[x] = e;
        fd.E32[x] = e32;
        E32_s[x] = e32;
    }
    // field energy sum by four full warps, one per SM sub-partition (FP64
    // instructions cost the same for any number of active lanes)
    constexpr int WE_THREADS = 128;
    double we = 0.0;
    if (threadIdx.x < WE_THREADS)
        for (int x = threadIdx.x; x < nx; x += WE_THREADS) we = fma(E_s[x], E_s[x], we);
    // field history (marker refinement): E of the state this kernel finishes
    if (fd.hist) {
        const long long slot = (count_step ? A->ctl->step + 1 : A->ctl->step) - fd.hist_origin;
        if (slot >= 0 && slot < fd.hist_cap)
            for (int x = threadIdx.x; x < nx; x += FIELD_THREADS) fd.hist[slot * nx + x] = E_s[x];
    }
    if (threadIdx.x < WE_THREADS) {
        for (int o = 16; o > 0; o >>= 1) we += __shfl_down_sync(0xffffffffu, we, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = we;
    }
    __syncthreads();
    // velocity rows the new field moves a marker in one step, per column
    // (used by the next step's deposit windows and finalize).  After a step
    // it replaces the previous step's table (the current one becomes the
    // previous); after a refresh it is the current table and the previous is 0.
    {
        Ctl* cw = A->ctl;
        __shared__ int smin_s[MAXS], smax_s[MAXS];
        if (threadIdx.x < MAXS) {
            smin_s[threadIdx.x] = 0x7fffffff;
            smax_s[threadIdx.x] = -0x7fffffff;
        }
        __syncthreads();
        for (int s = 0; s < A->ns; ++s) {
            const SpDev& sp = A->sp[s];
            // FP32: the table only places the deposit windows
            const float f = shf_s[s];
            const int tgt = tgt_s[s];
            int lmin = 0x7fffffff, lmax = -0x7fffffff;
            for (int x = threadIdx.x; x < nx; x += FIELD_THREADS) {
                float d = f * E32_s[x];
                d = d > 1.0e6f ? 1.0e6f : (d < -1.0e6f ? -1.0e6f : d);
                const int sh = isfinite(d) ? __float2int_rn(d) : 0;
                sp.shift[tgt][x] = sh;
                if (!count_step) sp.shift[1 - tgt][x] = 0;
                lmin = min(lmin, sh);
                lmax = max(lmax, sh);
            }
            lmin = __reduce_min_sync(0xffffffffu, lmin);
            lmax = __reduce_max_sync(0xffffffffu, lmax);
            if ((threadIdx.x & 31) == 0) {
                atomicMin(&smin_s[s], lmin);
                atomicMax(&smax_s[s], lmax);
            }
        }
        __syncthreads();
        if (threadIdx.x < A->ns) {
            const int q = threadIdx.x;
            const int tgt = tgt_s[q];
            cw->shift_min[q][tgt] = smin_s[q];
            cw->shift_max[q][tgt] = smax_s[q];
            if (!count_step) {
                cw->shift_min[q][1 - tgt] = 0;
                cw->shift_max[q][1 - tgt] = 0;
            }
        }
    }
    __syncthreads();
    __shared__ double WE_s;
    if (threadIdx.x == 0) {
        double s2 = 0.0;
        for (int w = 0; w < WE_THREADS / 32; ++w) s2 += red[w];
        WE_s = s2 * fd.we_scale;
    }
    // wait for the diagnostics sums, the re-sort decisions and the clearing by
    // the other CTAs, then write the diagnostics row and make this step's
    // markers and key counts current
    // warp 0, lane s: species s's control values that no other CTA of this
    // kernel writes, loaded before the barrier
    Ctl* ctl = A->ctl;
    const int ns = A->ns;
    const int s = threadIdx.x;
    const bool lane_sp = threadIdx.x < 32 && s < ns;
    unsigned long long ovf = 0, mv = 0, fm = 0;
    int sp_dim = 0, sp_mobile = 0, sp_nchunk = 0, sort_now = 0;
    long long sp_n = 0;
    if (lane_sp) {
        const SpDev& sp = A->sp[s];
        sp_dim = sp.nvdim;
        sp_mobile = sp.mobile;
        sp_nchunk = sp.nchunk;
        sp_n = sp.n;
        ovf = ctl->ovf_count[s];
        mv = ctl->movers[s];
        fm = ctl->far_movers[s];
        sort_now = ctl->sort_now[s];
    }
    cluster.sync();
    if (threadIdx.x < 32) {
        const double WE = WE_s;
        double N = 0.0, Wk = 0.0, S = 0.0;
        if (s < ns) {
            N = dfin[3 * s + 0];
            Wk = dfin[3 * s + 1];
            S = dfin[3 * s + 2];
            fd.diag[3 + s] = Wk;
            fd.diag[3 + ns + s] = N;
            fd.diag[3 + 2 * ns + s] = S;
        }
        const bool bad = __any_sync(0xffffffffu, s < ns && (!isfinite(N) || !isfinite(Wk) || !isfinite(S))) ||
                         !isfinite(WE);
        if (s == 0) {
            double wk_tot = 0.0;   // species order
            for (int q = 0; q < ns; ++q) wk_tot += dfin[3 * q + 1];
            fd.diag[0] = WE;
            fd.diag[1] = wk_tot;
            fd.diag[2] = WE + wk_tot;
            if (bad) ctl->err |= ERR_NUMERIC;
            if (count_step) ctl->step += 1;
        }
        if (s < ns) {
            ctl->ovf_last[s] = ovf;
            ctl->ovf_count[s] = 0;
            if (sp_dim == 3) {
                // 1d3v: the deposit just finalized becomes current, the other
                // accumulator (cleared by the finalize) takes the next one.
                // Re-sort when more than 1/64 of the markers sit off their
                // segment's row, or 1/4096 two or more rows off.
                const bool deposited = count_step ? sp_mobile != 0 : true;
                if (deposited) ctl->asel[s] ^= 1;
                ctl->movers[s] = 0;
                ctl->far_movers[s] = 0;
                if (count_step && sp_mobile) {
                    ctl->movers_last[s] = mv;
                    const unsigned long long n = (unsigned long long)sp_n;
                    const int so = (n > 0 && (mv * 64ull > n || fm * 4096ull > n)) ? 1 : 0;
                    ctl->sort_now[s] = so;
                    if (so) {
                        ctl->cur[s] = 1 - ctl->cur[s];
                        ctl->nsort[s] += 1;
                    }
                }
            } else if (count_step && sp_mobile && sp_nchunk > 0) {
                if (sort_now) {
                    ctl->cur[s] = 1 - ctl->cur[s];
                    ctl->nsort[s] += 1;
                }
                ctl->sort_now[s] = ctl->sort_next[s];
                ctl->hsel[s] = 1 - ctl->hsel[s];
                ctl->shsel[s] = 1 - ctl->shsel[s];
            }
        }
    }
}

// stand-alone field solve: one block, rho and E in global memory
__global__ void __launch_bounds__(FIELD_THREADS)
    k_poisson(const double* __restrict__ rho, double* __restrict__ E, int nx, int pow2,
              const double2* __restrict__ tw, const double* __restrict__ gmul)
{
    extern __shared__ __align__(16) unsigned char smem[];
    double* rho_s = reinterpret_cast<double*>(smem);
    double2* work = reinterpret_cast<double2*>(smem + poisson_rho_bytes(nx));
    double2* tw_s = reinterpret_cast<double2*>(smem + poisson_rho_bytes(nx) + poisson_work_bytes(nx));
    double* gm_s = reinterpret_cast<double*>(tw_s + nx / 2 + 1);
    const bool staged = poisson_stage(nx);
    if (staged) stage_tables(tw_s, gm_s, tw, gmul, nx);
    for (int x = threadIdx.x; x < nx; x += FIELD_THREADS) rho_s[x] = rho[x];
    __syncthreads();
    poisson_spectral(rho_s, work, staged ? tw_s : tw, staged ? gm_s : nullptr, nx, pow2, tw, gmul);
    for (int x = threadIdx.x; x < nx; x += FIELD_THREADS) E[x] = rho_s[x];
}

size_t poisson_smem_bytes(int nx) { return poisson_smem_bytes_dev(nx); }

void spectral_tables(int nx, double L, double cP, int softening, double2* tw, double* gm)
{
    const double dx = L / nx;
    for (int k = 0; k < nx; ++k) {
        const double a = 2.0 * M_PI * (double)k / (double)nx;
        tw[k] = make_double2(cos(a), -sin(a));
    }
    for (int m = 0; m <= nx / 2; ++m) gm[m] = 0.0;
    for (int m = 1; m <= nx / 2; ++m) {
        if (2 * m == nx) continue;   // Nyquist mode carries no field
        const double k = 2.0 * M_PI * (double)m / L;
        double kappa, K2;
        if (softening) {
            const double y1 = k * dx, y2 = 0.5 * k * dx;
            kappa = k * (sin(y1) / y1);
            K2 = k * k * (sin(y2) / y2) * (sin(y2) / y2);
        } else {
            kappa = k;
            K2 = k * k;
        }
        gm[m] = cP * kappa / K2;
    }
}

// Green's function of the spectral solve (Eq. 6): E_i = sum_j G[(i - j) mod nx]
// rho_j with G_n = (2 / nx) sum_m gm[m] sin(2 pi m n / nx) over the modes that
// carry a field (the multiplier -i gm[m] is odd in m, so the pairs (m, -m)
// give a sine; k = 0 and the Nyquist mode drop out).  Angles from exact
// integer indices (m n mod nx).
void green_table(int nx, const double* gm, double* G)
{
    std::vector<double> sn(nx);
    for (int k = 0; k < nx; ++k) sn[k] = sin(2.0 * M_PI * (double)k / (double)nx);
    for (int n = 0; n < nx; ++n) {
        double acc = 0.0;
        for (int m = 1; m <= nx / 2; ++m) acc += gm[m] * sn[(int)(((long long)m * n) % nx)];
        G[n] = 2.0 * acc / (double)nx;
    }
}

// The same solve as the circulant product with G, spread over many blocks
// (one warp per output, lanes over j, a fixed shuffle tree): FP64 work is
// spread over the SMs instead of one CTA's FFT.  rho, E, G: nx FP64 values.
__global__ void __launch_bounds__(256) k_poisson_dense(const double* __restrict__ rho, double* __restrict__ E, int nx,
                                                       const double* __restrict__ G)
{
    extern __shared__ __align__(16) unsigned char smem_d[];
    double* r = reinterpret_cast<double*>(smem_d);
    double* g = r + nx;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        r[i] = rho[i];
        g[i] = G[i];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = blockIdx.x * nw + warp; i < nx; i += gridDim.x * nw) {
        double acc = 0.0;
        for (int j = lane; j < nx; j += 32) {
            const int d = i - j;
            acc = fma(g[d < 0 ? d + nx : d], r[j], acc);
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) E[i] = acc;
    }
}

cudaError_t launch_poisson_dense(const double* rho, double* E, int nx, const double* G, cudaStream_t st)
{
    const int blocks = std::max(1, std::min((nx + 7) / 8, 148));
    k_poisson_dense<<<blocks, 256, (size_t)nx * 16, st>>>(rho, E, nx, G);
    return cudaGetLastError();
}

cudaError_t launch_poisson(const double* rho, double* E, int nx, const double2* tw, const double* gmul,
                           cudaStream_t st)
{
    const size_t smem = poisson_smem_bytes(nx);
    cudaError_t e = raise_smem_limit(k_poisson, (int)smem);
    if (e) return e;
    const int pow2 = poisson_pow2(nx) ? 1 : 0;
    k_poisson<<<1, FIELD_THREADS, smem, st>>>(rho, E, nx, pow2, tw, gmul);
    return cudaGetLastError();
}

// dynamic shared memory of the field kernel: the solve's (CTA 0)
size_t field_smem_bytes(const StepArgs& h) { return poisson_smem_bytes(h.fd.nx); }

cudaError_t configure_field_bytes(int bytes) { return raise_smem_limit(k_field, bytes); }

cudaError_t configure_field(const StepArgs& h) { return configure_field_bytes((int)field_smem_bytes(h)); }

cudaError_t launch_field(const StepArgs& h, const StepArgs* d, int count_step, cudaStream_t st)
{
    k_field<<<FIELD_CLUSTER, FIELD_THREADS, field_smem_bytes(h), st>>>(d, count_step, nullptr);
    return cudaGetLastError();
}


cudaError_t launch_field_batch(const BatchMap* bm, int nrun, int smem, int count_step, cudaStream_t st)
{
    if (nrun == 0) return cudaSuccess;
    k_field<<<FIELD_CLUSTER * nrun, FIELD_THREADS, smem, st>>>(nullptr, count_step, bm);
    return cudaGetLastError();
}

__global__ void k_log_table(double2* tab)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < LOG_TAB_N) {
        const double c = 1.0 + ((double)j + 0.5) / (double)LOG_TAB_N;
        tab[j] = make_double2(log(c), 1.0 / c);
    }
}

cudaError_t init_log_table(double2* tab, cudaStream_t st)
{
    k_log_table<<<(LOG_TAB_N + 255) / 256, 256, 0, st>>>(tab);
    return cudaGetLastError();
}

}  // namespace avl
