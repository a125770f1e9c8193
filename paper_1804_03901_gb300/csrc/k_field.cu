// k_field.cu -- net charge density and spectral Poisson solve (Sec. 3.1,
// Eq. 5 / Eq. 6a-c), diagnostics row (Sec. 3.4.1) and the re-sort decision.
//
// One thread-block cluster of FIELD_CLUSTER CTAs.  Every CTA sums the charge
// partials of a slice of x over all species and velocity row blocks and
// writes its slice into CTA 0's shared memory (distributed shared memory);
// CTA 0 then runs an FP64 real FFT of length nx (a complex radix-2 FFT of
// length nx/2 with the even/odd split), multiplies by -i cP kappa / K^2,
// transforms back, and writes E in FP64 and FP32.  A direct DFT serves grid
// sizes that are not a power of two.
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

// in-place radix-2 decimation-in-time FFT of length M (power of two) on
// shared memory, input already in bit-reversed order; tw[k] = exp(-2 pi i k/N)
// with N = 2 M; inverse uses the conjugate twiddles (no scaling).
__device__ void fft_pow2(double2* a, int M, int N, const double2* __restrict__ tw, bool inverse)
{
    for (int len = 2; len <= M; len <<= 1) {
        const int half = len >> 1;
        const int step = N / len;
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

// Spectral Poisson solve (Eq. 5 / Eq. 6a-c) by the whole block: rho_s holds
// rho in shared memory (nx doubles, overwritten), work is shared scratch of
// nx/2 + 2 complex values; tw[k] = exp(-2 pi i k / nx), gmul[m] = cP kappa_m /
// K2_m (zero at m = 0 and at the Nyquist mode).  Writes E (nx) to Eout.
__device__ void poisson_spectral(double* rho_s, double2* work, double* Eout, int nx, int pow2,
                                 const double2* __restrict__ tw, const double* __restrict__ gmul)
{
    if (pow2) {
        const int M = nx / 2;
        int bits = 0;
        while ((1 << bits) < M) ++bits;
        for (int n = threadIdx.x; n < M; n += FIELD_THREADS)
            work[bitrev(n, bits)] = make_double2(rho_s[2 * n], rho_s[2 * n + 1]);
        __syncthreads();
        fft_pow2(work, M, nx, tw, false);
        // unpack X_m = Ev_m + W^m Od_m and form Ehat_m = -i g_m X_m  (m = 0..M)
        // then pack Y_m = Ev'_m + i Od'_m of the field for the inverse.
        double2* Y = reinterpret_cast<double2*>(rho_s);   // reuse: needs M * 16 = nx * 8 bytes
        // compute Ehat into registers per m, then pair (m, M - m)
        for (int m = threadIdx.x; m < M; m += FIELD_THREADS) {
            // X_m and X_{M-m}
            const double2 Zm = work[m];
            const double2 Zc = conj2(work[(M - m) % M]);
            const double2 ev = make_double2(0.5 * (Zm.x + Zc.x), 0.5 * (Zm.y + Zc.y));
            const double2 dd = make_double2(0.5 * (Zm.x - Zc.x), 0.5 * (Zm.y - Zc.y));   // = i Od
            const double2 od = make_double2(dd.y, -dd.x);                                 // Od = -i dd
            const double2 Xm = cadd(ev, cmul(tw[m], od));
            // partner index p = M - m (for m = 0 the partner is the Nyquist mode M)
            const int mp = M - m;
            const double2 Zp = work[mp % M];
            const double2 Zpc = conj2(work[m]);   // Z_{M - mp} = Z_m
            const double2 evp = make_double2(0.5 * (Zp.x + Zpc.x), 0.5 * (Zp.y + Zpc.y));
            const double2 ddp = make_double2(0.5 * (Zp.x - Zpc.x), 0.5 * (Zp.y - Zpc.y));
            const double2 odp = make_double2(ddp.y, -ddp.x);
            double2 twp = (mp < nx) ? tw[mp] : make_double2(1.0, 0.0);
            const double2 Xp = cadd(evp, cmul(twp, odp));
            // Ehat = -i g X  ->  (g X.y, -g X.x)
            const double gm = gmul[m], gp = gmul[mp];
            const double2 Em = make_double2(gm * Xm.y, -gm * Xm.x);
            const double2 Ep = make_double2(gp * Xp.y, -gp * Xp.x);
            // inverse pack: Ev'_m = (E_m + conj(E_{M-m}))/2, Od'_m = (E_m - conj(E_{M-m}))/2 * exp(+2 pi i m/N)
            const double2 Epc = conj2(Ep);
            const double2 ev2 = make_double2(0.5 * (Em.x + Epc.x), 0.5 * (Em.y + Epc.y));
            const double2 od2 = cmul(make_double2(0.5 * (Em.x - Epc.x), 0.5 * (Em.y - Epc.y)), conj2(tw[m]));
            Y[bitrev(m, bits)] = make_double2(ev2.x - od2.y, ev2.y + od2.x);   // ev2 + i od2
        }
        __syncthreads();
        fft_pow2(Y, M, nx, tw, true);
        const double inv = 1.0 / (double)M;
        for (int n = threadIdx.x; n < M; n += FIELD_THREADS) {
            const double2 y = Y[n];
            Eout[2 * n] = y.x * inv;
            Eout[2 * n + 1] = y.y * inv;
        }
    } else {
        // direct DFT: Ehat_m for m = 1 .. (nx-1)/2, then E_i = (2/N) sum Re(Ehat_m e^{+i})
        const int mmax = (nx - 1) / 2;
        for (int m = 1 + threadIdx.x; m <= mmax; m += FIELD_THREADS) {
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
        for (int i = threadIdx.x; i < nx; i += FIELD_THREADS) {
            double acc = 0.0;
            for (int m = 1; m <= mmax; ++m) {
                const double2 w = tw[(int)(((long long)m * i) % nx)];
                // Re(E_m * conj(w))
                acc += work[m].x * w.x + work[m].y * w.y;
            }
            Eout[i] = 2.0 * acc / (double)nx;
        }
    }
}

// Markers a chunk's best deposit window holds: the largest sum of wk
// consecutive bins of its HIST_S-bin key histogram (the window best_window
// places).  Called by a whole warp; one coalesced load and a warp scan.
__device__ int best_cover_warp(const int* __restrict__ hist, int wk)
{
    static_assert(HIST_S == 64, "two bins per lane");
    const int lane = threadIdx.x & 31;
    const int2 h = reinterpret_cast<const int2*>(hist)[lane];
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
__device__ void resort_work(const StepArgs* __restrict__ A, int rank)
{
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
        // markers outside the best window of their chunk (a warp per chunk)
        if (threadIdx.x == 0) miss = 0;
        __syncthreads();
        const int wk = max(1, min(HIST_S, sp.Wmax - 2 * HALO - 1));
        unsigned long long my = 0;
        for (int c = threadIdx.x >> 5; c < sp.nchunk; c += FIELD_THREADS / 32) {
            const int covered = best_cover_warp(cnt + (size_t)c * HIST_S, wk);
            const int beg = c * sp.M;
            const int end = (int)min((long long)(c + 1) * sp.M, sp.n);
            if ((threadIdx.x & 31) == 0) my += (unsigned long long)((end - beg) - covered);
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
            scan_layout(sp, kref, cnt, far, true, sp.KB[1 - cur_after]);
            // the next step deposits from the re-sorted layout: its window
            // placement takes the key histograms of the re-sorted chunks
            sorted_chunk_hist(sp, sp.KB[1 - cur_after], sp.cnt[1 - hs]);
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
    double* rho_s = reinterpret_cast<double*>(smem);                 // nx
    double2* work = reinterpret_cast<double2*>(smem + ((size_t)nx * 8 + 15) / 16 * 16);   // nx/2 + 1
    __shared__ double red[FIELD_THREADS / 32];
    __shared__ double dfin[3 * MAXS];   // per-species diagnostics sums (written by CTA FIELD_DIAG)

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
        if (count_step) resort_work(A, rank);
        cluster.sync();
        return;
    }

    // --- CTA 0: Poisson --------------------------------------------------
    for (int x = threadIdx.x; x < nx; x += FIELD_THREADS) fd.rho[x] = rho_s[x];
    double* Eout = fd.E64;
    poisson_spectral(rho_s, work, Eout, nx, fd.pow2, fd.tw, fd.gmul);
    __syncthreads();
    // --- E in FP32, field energy, diagnostics row --------------------------
    double we = 0.0;
    for (int x = threadIdx.x; x < nx; x += FIELD_THREADS) {
        const double e = Eout[x];
        fd.E32[x] = (float)e;
        we += e * e;
    }
    // field history (marker refinement): E of the state this kernel finishes
    if (fd.hist) {
        const long long slot = (count_step ? A->ctl->step + 1 : A->ctl->step) - fd.hist_origin;
        if (slot >= 0 && slot < fd.hist_cap)
            for (int x = threadIdx.x; x < nx; x += FIELD_THREADS) fd.hist[slot * nx + x] = Eout[x];
    }
    for (int o = 16; o > 0; o >>= 1) we += __shfl_down_sync(0xffffffffu, we, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = we;
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
            const double f = sp.mobile ? sp.qm_dt * sp.inv_dv[0] : 0.0;
            const int tgt = count_step ? 1 - cw->shsel[s] : cw->shsel[s];
            int lmin = 0x7fffffff, lmax = -0x7fffffff;
            for (int x = threadIdx.x; x < nx; x += FIELD_THREADS) {
                double d = f * Eout[x];
                d = d > 1.0e6 ? 1.0e6 : (d < -1.0e6 ? -1.0e6 : d);
                const int sh = isfinite(d) ? (int)rint(d) : 0;
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
            const int tgt = count_step ? 1 - cw->shsel[q] : cw->shsel[q];
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
        for (int w = 0; w < FIELD_THREADS / 32; ++w) s2 += red[w];
        WE_s = s2 * fd.dx / (2.0 * fd.cP);
    }
    // wait for the diagnostics sums, the re-sort decisions and the clearing by
    // the other CTAs, then write the diagnostics row and make this step's
    // markers and key counts current
    cluster.sync();
    if (threadIdx.x == 0) {
        Ctl* ctl = A->ctl;
        const int ns = A->ns;
        const double WE = WE_s;
        double wk_tot = 0.0;
        bool bad = !isfinite(WE);
        for (int s = 0; s < ns; ++s) {
            const double N = dfin[3 * s + 0], Wk = dfin[3 * s + 1], S = dfin[3 * s + 2];
            fd.diag[3 + s] = Wk;
            fd.diag[3 + ns + s] = N;
            fd.diag[3 + 2 * ns + s] = S;
            wk_tot += Wk;
            bad = bad || !isfinite(N) || !isfinite(Wk) || !isfinite(S);
        }
        fd.diag[0] = WE;
        fd.diag[1] = wk_tot;
        fd.diag[2] = WE + wk_tot;
        if (bad) ctl->err |= ERR_NUMERIC;
        for (int s = 0; s < ns; ++s) {
            ctl->ovf_last[s] = ctl->ovf_count[s];
            ctl->ovf_count[s] = 0;
        }
        for (int s = 0; s < ns; ++s) {
            const SpDev& sp = A->sp[s];
            if (sp.nvdim == 3) {
                // 1d3v: the deposit just finalized becomes current, the other
                // accumulator (cleared by the finalize) takes the next one.
                // Re-sort when more than 1/64 of the markers sit off their
                // segment's row, or 1/4096 two or more rows off.
                const bool deposited = count_step ? sp.mobile != 0 : true;
                if (deposited) ctl->asel[s] ^= 1;
                const unsigned long long mv = ctl->movers[s], fm = ctl->far_movers[s];
                ctl->movers[s] = 0;
                ctl->far_movers[s] = 0;
                if (count_step && sp.mobile) {
                    ctl->movers_last[s] = mv;
                    const unsigned long long n = (unsigned long long)sp.n;
                    const int so = (n > 0 && (mv * 64ull > n || fm * 4096ull > n)) ? 1 : 0;
                    ctl->sort_now[s] = so;
                    if (so) {
                        ctl->cur[s] = 1 - ctl->cur[s];
                        ctl->nsort[s] += 1;
                    }
                }
                continue;
            }
            if (!count_step) continue;
            if (!sp.mobile || sp.nchunk == 0) continue;
            if (ctl->sort_now[s]) {
                ctl->cur[s] = 1 - ctl->cur[s];
                ctl->nsort[s] += 1;
            }
            ctl->sort_now[s] = ctl->sort_next[s];
            ctl->hsel[s] = 1 - ctl->hsel[s];
            ctl->shsel[s] = 1 - ctl->shsel[s];
        }
        if (count_step) ctl->step += 1;
    }
}

// stand-alone field solve: one block, rho and E in global memory
__global__ void __launch_bounds__(FIELD_THREADS)
    k_poisson(const double* __restrict__ rho, double* __restrict__ E, int nx, int pow2,
              const double2* __restrict__ tw, const double* __restrict__ gmul)
{
    extern __shared__ __align__(16) unsigned char smem[];
    double* rho_s = reinterpret_cast<double*>(smem);
    double2* work = reinterpret_cast<double2*>(smem + ((size_t)nx * 8 + 15) / 16 * 16);
    for (int x = threadIdx.x; x < nx; x += FIELD_THREADS) rho_s[x] = rho[x];
    __syncthreads();
    poisson_spectral(rho_s, work, E, nx, pow2, tw, gmul);
}

size_t poisson_smem_bytes(int nx) { return ((size_t)nx * 8 + 15) / 16 * 16 + ((size_t)nx / 2 + 2) * 16; }

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
    const int pow2 = (nx >= 4 && (nx & (nx - 1)) == 0) ? 1 : 0;
    k_poisson<<<1, FIELD_THREADS, smem, st>>>(rho, E, nx, pow2, tw, gmul);
    return cudaGetLastError();
}

static size_t field_smem(const StepArgs& h)
{
    const int nx = h.fd.nx;
    return ((size_t)nx * 8 + 15) / 16 * 16 + ((size_t)nx / 2 + 2) * 16;
}

cudaError_t configure_field_bytes(int bytes) { return raise_smem_limit(k_field, bytes); }

cudaError_t configure_field(const StepArgs& h) { return configure_field_bytes((int)field_smem(h)); }

cudaError_t launch_field(const StepArgs& h, const StepArgs* d, int count_step, cudaStream_t st)
{
    k_field<<<FIELD_CLUSTER, FIELD_THREADS, field_smem(h), st>>>(d, count_step, nullptr);
    return cudaGetLastError();
}

size_t field_smem_bytes(int nx) { return ((size_t)nx * 8 + 15) / 16 * 16 + ((size_t)nx / 2 + 2) * 16; }

cudaError_t launch_field_batch(const BatchMap* bm, int nrun, int smem, int count_step, cudaStream_t st)
{
    if (nrun == 0) return cudaSuccess;
    k_field<<<FIELD_CLUSTER * nrun, FIELD_THREADS, smem, st>>>(nullptr, count_step, bm);
    return cudaGetLastError();
}

}  // namespace avl
