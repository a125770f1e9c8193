// k_vhs1.cu -- 1d1v kernels of the Vlasov-Hybrid time step (Fig. 2).
//
// One step of one species runs as
//   k_rs1      only on steps the field kernel marked for re-sorting: every
//              marker into its slot of the layout sorted by its current key,
//              in the other buffer
//   k_pd1      per chunk: gather E + push (Sec. 2), VHS deposit of the
//              numerator and denominator of Eq. 4 into a shared-memory window
//              (runs of markers with the same cloud-in-cell footprint are
//              summed in registers first), the pushed markers written back in
//              place and their new keys counted
//   k_fin1     f = num / den (Eq. 4), velocity moment (Eq. 14), per-block
//              diagnostics (Sec. 3.4.1)
// k_count1 counts the keys of freshly created markers.  Marker creation
// (lattice weighted to f0, Sec. 2 / Sec. 3.1) and caller markers go through
// a count / scan / scatter of their own.
#include <math.h>

#include <algorithm>

#include "avl_internal.cuh"
#include "common.cuh"
#include "ptx.cuh"
#include "resort.cuh"

namespace avl {

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
// n / M for 0 <= n < 2^31 by a multiply-high (magic m, shift l from the host)
__device__ __forceinline__ int chunk_of(int n, unsigned m, int l)
{
    return (int)(__umulhi((unsigned)n, m) >> (l - 1));
}

__device__ __forceinline__ int species_of_chunk(const StepArgs* A, int g)
{
    int s = 0;
    while (s + 1 < A->ns && g >= A->sp[s + 1].chunk_base) ++s;
    return s;
}

__device__ __forceinline__ int species_of_fin(const StepArgs* A, int g)
{
    int s = 0;
    while (s + 1 < A->ns && g >= A->sp[s + 1].fin_base) ++s;
    return s;
}

// key = lower velocity row of the cloud-in-cell footprint ("dual row"),
// clamped to [0, nv).  Explicit fused multiply-add so that every kernel
// computes bit-identical keys.
__device__ __forceinline__ int key_rel(float dv, int kb, float inv_dv, int nv)
{
    return clampi(kb + (int)floorf(__fmaf_rn(dv, inv_dv, -0.5f)), 0, nv - 1);
}
__device__ __forceinline__ int key_rel(double dv, int kb, double inv_dv, int nv)
{
    return clampi(kb + (int)floor(__fma_rn(dv, inv_dv, -0.5)), 0, nv - 1);
}
__device__ __forceinline__ int key_abs(double v, double vmin, double inv_dv, int nv)
{
    const double t = __fma_rn(__dsub_rn(v, vmin), inv_dv, -0.5);
    if (!(t > -4.0e9 && t < 4.0e9)) return t > 0 ? nv - 1 : 0;
    return clampi((int)floor(t), 0, nv - 1);
}


// MPT consecutive values from an aligned address (marker arrays are padded to
// a multiple of 64 entries, so a group starting below n is in bounds)
__device__ __forceinline__ void loadg(const float* p, float (&o)[4])
{
    const float4 a = *reinterpret_cast<const float4*>(p);
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
}
__device__ __forceinline__ void loadg(const int* p, int (&o)[4])
{
    const int4 a = *reinterpret_cast<const int4*>(p);
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
}
__device__ __forceinline__ void loadg(const double* p, double (&o)[4])
{
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void loadg(const long long* p, long long (&o)[4])
{
    const longlong2 a = reinterpret_cast<const longlong2*>(p)[0], b = reinterpret_cast<const longlong2*>(p)[1];
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void storeg(float* p, const float (&o)[4])
{
    *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
}
__device__ __forceinline__ void storeg(int* p, const int (&o)[4])
{
    *reinterpret_cast<int4*>(p) = make_int4(o[0], o[1], o[2], o[3]);
}
__device__ __forceinline__ void storeg(double* p, const double (&o)[4])
{
    reinterpret_cast<double2*>(p)[0] = make_double2(o[0], o[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(o[2], o[3]);
}
__device__ __forceinline__ void storeg(long long* p, const long long (&o)[4])
{
    reinterpret_cast<longlong2*>(p)[0] = make_longlong2(o[0], o[1]);
    reinterpret_cast<longlong2*>(p)[1] = make_longlong2(o[2], o[3]);
}
// eight consecutive values (count kernel)
__device__ __forceinline__ void load8(const float* p, float (&o)[8])
{
    const float4 a = *reinterpret_cast<const float4*>(p), b = *reinterpret_cast<const float4*>(p + 4);
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
}
__device__ __forceinline__ void load8(const int* p, int (&o)[8])
{
    const int4 a = *reinterpret_cast<const int4*>(p), b = *reinterpret_cast<const int4*>(p + 4);
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
}
__device__ __forceinline__ void load8(const double* p, double (&o)[8])
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const double2 a = reinterpret_cast<const double2*>(p)[q];
        o[2 * q] = a.x;
        o[2 * q + 1] = a.y;
    }
}
__device__ __forceinline__ void store8(float* p, const float (&o)[8])
{
    reinterpret_cast<float4*>(p)[0] = make_float4(o[0], o[1], o[2], o[3]);
    reinterpret_cast<float4*>(p)[1] = make_float4(o[4], o[5], o[6], o[7]);
}
__device__ __forceinline__ void store8(int* p, const int (&o)[8])
{
    reinterpret_cast<int4*>(p)[0] = make_int4(o[0], o[1], o[2], o[3]);
    reinterpret_cast<int4*>(p)[1] = make_int4(o[4], o[5], o[6], o[7]);
}
__device__ __forceinline__ void store8(double* p, const double (&o)[8])
{
#pragma unroll
    for (int q = 0; q < 4; ++q) reinterpret_cast<double2*>(p)[q] = make_double2(o[2 * q], o[2 * q + 1]);
}

// periodic neighbours of a lower cloud-in-cell cell i0, which is in
// [-1, nx - 1] for every stored position (cell in [0, nx), offset in
// [0, 1)); any other value still maps into the grid
__device__ __forceinline__ void wrap_pair_in(int i0, int nx, int& ia, int& ib)
{
    ia = (unsigned)i0 < (unsigned)nx ? i0 : nx - 1;
    ib = (unsigned)(i0 + 1) < (unsigned)nx ? i0 + 1 : 0;
}

// numerator and denominator contributions of a run of markers that share the
// same four cells (lower corner i0, j0)
template <typename T>
struct Run;

// FP32: a run holds at most MPT markers, summed in registers; the run sums
// are added into the window with plain FP32 shared-memory reductions.  The
// window's numerator plane holds deviations from a reference value per
// cell, sum alpha (f_l - f_ref), with f_ref the cell's f of the previous
// reconstruction (staged in shared memory beside the window); the finalize
// forms f = f_ref + sum alpha (f_l - f_ref) / sum alpha, which is Eq. 4 for
// any f_ref.  A run sums alpha (f_l - r) about the value r of its first
// marker and shifts the sum to each cell's reference when it is flushed,
// fma(r - f_ref, sum alpha, sum alpha (f_l - r)), so that every rounding of
// the numerator (products, register sums, window sums) scales with the
// spread of the marker values in the cell and the change of f since the
// previous reconstruction (a few per cent of f for a smooth f) instead of
// with f itself; the rounding of the denominator enters f only through
// (f - f_ref) as well.  Runs outside the window carry absolute values into
// the FP64 overflow grids.
template <>
struct Run<float> {
    int i0, j0;
    float r;
    float nh[4], dh[4];
    __device__ __forceinline__ void reset(int i, int j)
    {
        i0 = i;
        j0 = j;
        r = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) nh[k] = dh[k] = 0.f;
    }
    __device__ __forceinline__ void add(const float (&a)[4], float f, bool first)
    {
        if (first) r = f;
        const float d = __fsub_rn(f, r);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            nh[k] = __fmaf_rn(a[k], d, nh[k]);
            dh[k] = __fadd_rn(dh[k], a[k]);
        }
    }
    // window planes: num (deviations from fref), den
    __device__ __forceinline__ void to_window(float* win, int plane, const int (&cell)[4], const float* fref) const
    {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            atomicAdd(win + cell[k], __fmaf_rn(__fsub_rn(r, fref[cell[k]]), dh[k], nh[k]));
            atomicAdd(win + plane + cell[k], dh[k]);
        }
    }
    // absolute sums (overflow path, FP64)
    __device__ __forceinline__ double num(int k) const { return (double)nh[k] + (double)r * (double)dh[k]; }
    __device__ __forceinline__ double den(int k) const { return (double)dh[k]; }
};

template <>
struct Run<double> {
    int i0, j0;
    double nh[4], dh[4];
    __device__ __forceinline__ void reset(int i, int j)
    {
        i0 = i;
        j0 = j;
#pragma unroll
        for (int k = 0; k < 4; ++k) nh[k] = dh[k] = 0.0;
    }
    __device__ __forceinline__ void add(const double (&a)[4], double f, bool)
    {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            nh[k] += a[k] * f;
            dh[k] += a[k];
        }
    }
    // window planes: num, den
    __device__ __forceinline__ void to_window(double* win, int plane, const int (&cell)[4], const double*) const
    {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            atomicAdd(win + cell[k], nh[k]);
            atomicAdd(win + plane + cell[k], dh[k]);
        }
    }
    __device__ __forceinline__ double num(int k) const { return nh[k]; }
    __device__ __forceinline__ double den(int k) const { return dh[k]; }
};

// the rare out-of-window path: FP64 global atomics into the overflow grids;
// each row written is tagged with the step (tag), so that the finalize reads
// and clears only the rows of this step's overflow
__device__ __forceinline__ void flush_overflow(int ia, int ib, int j0, int nx, int nv, double n0, double n1, double n2,
                                            double n3, double d0, double d1, double d2, double d3,
                                            double* ovf_num, double* ovf_den, int* ovf_tag, int tag)
{
    if (j0 >= 0 && j0 < nv) {
        const size_t o = (size_t)j0 * nx;
        atomicAdd(ovf_num + o + ia, n0);
        atomicAdd(ovf_den + o + ia, d0);
        atomicAdd(ovf_num + o + ib, n1);
        atomicAdd(ovf_den + o + ib, d1);
        ovf_tag[j0] = tag;
    }
    if (j0 + 1 >= 0 && j0 + 1 < nv) {
        const size_t o = (size_t)(j0 + 1) * nx;
        atomicAdd(ovf_num + o + ia, n2);
        atomicAdd(ovf_den + o + ia, d2);
        atomicAdd(ovf_num + o + ib, n3);
        atomicAdd(ovf_den + o + ib, d3);
        ovf_tag[j0 + 1] = tag;
    }
}

// flush a run into the window or, if one of its rows falls outside, into the
// FP64 overflow grids; window row of grid row j at column x = j - sh[x] - row0.
// Returns true for the overflow path.
template <typename T>
__device__ __forceinline__ bool flush_run(const Run<T>& r, T* win, int plane, int row0, int W, int nx, int nv,
                                          const int* sh, const T* fref, double* ovf_num, double* ovf_den,
                                          int* ovf_tag, int tag)
{
    if (r.j0 + 1 < 0 || r.j0 >= nv) return false;   // footprint entirely off the velocity grid
    int ia, ib;
    wrap_pair_in(r.i0, nx, ia, ib);
    const int wa = r.j0 - sh[ia] - row0, wb = r.j0 - sh[ib] - row0;
    if (wa >= 0 && wa + 1 < W && wb >= 0 && wb + 1 < W) {
        const int cell[4] = {wa * nx + ia, wb * nx + ib, (wa + 1) * nx + ia, (wb + 1) * nx + ib};
        r.to_window(win, plane, cell, fref);
        return false;
    }
    flush_overflow(ia, ib, r.j0, nx, nv, r.num(0), r.num(1), r.num(2), r.num(3), r.den(0), r.den(1), r.den(2),
                   r.den(3), ovf_num, ovf_den, ovf_tag, tag);
    return true;
}

// one chunk's deposit window: numerator and denominator planes of Wmax rows
size_t window_bytes(const SpDev& sp, int prec)
{
    return (size_t)2 * (prec == AVL_FP32 ? 4 : 8) * win_plane(sp.Wmax, sp.nx);
}

// the FP32 reference plane (f of the previous reconstruction over the window)
static size_t fref_bytes(const SpDev& sp, int prec)
{
    return prec == AVL_FP32 ? (size_t)4 * win_plane(sp.Wmax, sp.nx) : 0;
}

size_t pd1_smem_bytes(const SpDev& sp, int prec)
{
    size_t eb = (size_t)sp.nx * (prec == AVL_FP32 ? 4 : 8);
    eb = (eb + 15) & ~size_t(15);
    return eb + 32 + (size_t)2 * HIST_S * 4 + (((size_t)4 * sp.nx + 15) & ~size_t(15)) + window_bytes(sp, prec) +
           fref_bytes(sp, prec);
}

// ---------------------------------------------------------------------------
// slot assignment within a warp
// ---------------------------------------------------------------------------
// Every lane holds up to MPT consecutive markers with key codes code[m]
// (-1: no marker), lanes in storage order.  For every key the warp's markers
// get consecutive slots in storage order, starting at the chunk's first slot
// for that key offs[code] (global) plus the chunk's running count scnt[code]
// (shared); so a thread's run of same-key markers stays together.  Far keys
// (code >= HIST_S) take slots from the global per-key cursor far_cur.
__device__ __forceinline__ void assign_slots(const int (&code)[MPT], int* scnt, const int* __restrict__ offs,
                                             int* far_cur, int (&dst)[MPT])
{
    const int lane = threadIdx.x & 31;
    // common case: every lane holds MPT markers of one in-histogram key
    {
        const int k0 = code[0];
        bool same = k0 >= 0 && k0 < HIST_S;
#pragma unroll
        for (int m = 1; m < MPT; ++m) same = same && code[m] == k0;
        const int kw = __shfl_sync(0xffffffffu, k0, 0);
        if (__all_sync(0xffffffffu, same && k0 == kw)) {
            int base = 0;
            if (lane == 0) base = offs[kw] + atomicAdd(scnt + kw, 32 * MPT);
            base = __shfl_sync(0xffffffffu, base, 0) + lane * MPT;
#pragma unroll
            for (int m = 0; m < MPT; ++m) dst[m] = base + m;
            return;
        }
    }
    unsigned done = 0;
#pragma unroll
    for (int m = 0; m < MPT; ++m) {
        dst[m] = -1;
        if (code[m] < 0) done |= 1u << m;
    }
    for (int guard = 0; guard < 32 * MPT + 1; ++guard) {
        int mine = 0x7fffffff;
#pragma unroll
        for (int m = 0; m < MPT; ++m)
            if (!(done >> m & 1)) mine = min(mine, code[m]);
        const int k = __reduce_min_sync(0xffffffffu, mine);
        if (k == 0x7fffffff) break;
        int n = 0;
#pragma unroll
        for (int m = 0; m < MPT; ++m) n += (!(done >> m & 1) && code[m] == k) ? 1 : 0;
        int incl = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        int base = 0;
        if (lane == 0) base = (k >= HIST_S) ? atomicAdd(far_cur + (k - HIST_S), total) : offs[k] + atomicAdd(scnt + k, total);
        base = __shfl_sync(0xffffffffu, base, 0);
        int d = base + incl - n;
#pragma unroll
        for (int m = 0; m < MPT; ++m) {
            if (!(done >> m & 1) && code[m] == k) {
                dst[m] = d++;
                done |= 1u << m;
            }
        }
    }
}

// warp-aggregated histogram of key codes: codes < HIST_S into the shared
// histogram, far codes into the global per-key counts
__device__ __forceinline__ void hist_add(int* hist, int* far_cnt, int code, bool valid)
{
    const int key = valid ? code : -1;
    const unsigned mask = __match_any_sync(0xffffffffu, key);
    const int lane = threadIdx.x & 31;
    if (valid && lane == __ffs(mask) - 1) {
        if (code < HIST_S)
            atomicAdd(hist + code, __popc(mask));
        else
            atomicAdd(far_cnt + (code - HIST_S), __popc(mask));
    }
}

// ---------------------------------------------------------------------------
// key histograms of the current markers (after marker creation; one CTA per chunk)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(CNT_THREADS) k_count1(const StepArgs* __restrict__ A)
{
    __shared__ int hist[HIST_S];
    const int g = blockIdx.x;
    const int s = species_of_chunk(A, g);
    const SpDev& sp = A->sp[s];
    Ctl* ctl = A->ctl;
    const int c = g - sp.chunk_base;
    const int hs = ctl->hsel[s];
    const int cb = ctl->cur[s];
    const int kb = sp.KB[cb][c];
    const int kbase = kb - HIST_R;
    const int beg = c * sp.M, end = (int)min((long long)(c + 1) * sp.M, sp.n);
    for (int i = threadIdx.x; i < HIST_S; i += CNT_THREADS) hist[i] = 0;
    __syncthreads();
    const T* dvp = reinterpret_cast<const T*>(sp.mv[cb][0]);
    const T inv_dv = (T)sp.inv_dv[0];
    const int nv = sp.nvflat;
    for (int b0 = beg; b0 < end; b0 += CNT_THREADS * 8) {
        const int g0 = b0 + threadIdx.x * 8;
        T d8[8];
        if (g0 < end) load8(dvp + g0, d8);
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const bool ok = g0 + m < end;
            const int key = ok ? key_rel(d8[m], kb, inv_dv, nv) : 0;
            hist_add(hist, sp.far_cnt[hs], rel_code(key, kbase), ok);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < HIST_S; i += CNT_THREADS) sp.cnt[hs][(size_t)c * HIST_S + i] = hist[i];
}

// ---------------------------------------------------------------------------
// re-sort (one CTA per chunk): markers into the layout sorted by their keys
// ---------------------------------------------------------------------------
// On a step the field kernel marked for re-sorting, every marker of the chunk
// goes, before the push, to its slot of the layout sorted by its current key
// (slots prepared by the field kernel from the key counts of the current
// state) in the other buffer, with its velocity re-referenced to the target
// chunk.  The push + deposit kernel then works in place on that buffer.
constexpr int RS_ROUNDS = 4;       // 32-marker rounds per warp and tile of the re-sort
constexpr int RS_KB_SMEM = 4096;   // reference keys of the target chunks staged in shared memory

template <typename T, bool BATCH>
__global__ void __launch_bounds__(PD_THREADS) k_rs1(const StepArgs* __restrict__ A0, const BatchMap* __restrict__ bm)
{
    __shared__ int scnt[HIST_S], offs_s[HIST_S];
    __shared__ int kbn_s[RS_KB_SMEM];
    __shared__ int nbad_s;
    int g = blockIdx.x;
    const StepArgs* __restrict__ A = A0;
    if constexpr (BATCH) A = batch_run(A0, bm, bm->pd_base, g);
    const int s = species_of_chunk(A, g);
    const SpDev& sp = A->sp[s];
    Ctl* ctl = A->ctl;
    if (!sp.mobile || !ctl->sort_now[s]) return;
    const int c = g - sp.chunk_base;
    const int cb = ctl->cur[s], nb = 1 - cb;
    const int n_all = (int)sp.n;
    const int nv = sp.nvflat;
    const int beg = c * sp.M, end = min((c + 1) * sp.M, n_all);
    const int kb = sp.KB[cb][c];
    const int kbase = kb - HIST_R;
    const int* kb_new_g = sp.KB[nb];
    const bool kb_in_smem = sp.nchunk <= RS_KB_SMEM;
    for (int i = threadIdx.x; i < HIST_S; i += PD_THREADS) {
        scnt[i] = 0;
        offs_s[i] = sp.offs[(size_t)c * HIST_S + i];
    }
    if (kb_in_smem)
        for (int i = threadIdx.x; i < sp.nchunk; i += PD_THREADS) kbn_s[i] = kb_new_g[i];
    if (threadIdx.x == 0) nbad_s = 0;
    __syncthreads();
    const int* kb_new = kb_in_smem ? kbn_s : kb_new_g;
    const T inv_dv = (T)sp.inv_dv[0];
    const T dvk = (T)sp.dv[0];
    const T* dvp = reinterpret_cast<const T*>(sp.mv[cb][0]);
    const T* fp = reinterpret_cast<const T*>(sp.mf[cb]);
    T* dvp_out = reinterpret_cast<T*>(sp.mv[nb][0]);
    T* fp_out = reinterpret_cast<T*>(sp.mf[nb]);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    int n_bad = 0;
    // a tile: every warp takes RS_ROUNDS x 32 consecutive markers, lane l the
    // l-th of each round, so that a round's slots (warp-aggregated per key,
    // in storage order) and its stores are contiguous
    constexpr int TILE = PD_THREADS * RS_ROUNDS;
    for (int tb = beg; tb < end; tb += TILE) {
        const int w0 = tb + warp * 32 * RS_ROUNDS;
        T dv[RS_ROUNDS], f[RS_ROUNDS];
        PosM<T> pos[RS_ROUNDS];
#pragma unroll
        for (int r = 0; r < RS_ROUNDS; ++r) {
            const int i = w0 + r * 32 + lane;
            if (i < end) {
                dv[r] = dvp[i];
                f[r] = fp[i];
                pos[r].load(sp, cb, i);
            } else {
                dv[r] = (T)0;
                f[r] = (T)0;
            }
        }
#pragma unroll
        for (int r = 0; r < RS_ROUNDS; ++r) {
            const int i = w0 + r * 32 + lane;
            const bool ok = i < end;
            const int code = ok ? rel_code(key_rel(dv[r], kb, inv_dv, nv), kbase) : -1;
            const unsigned grp = __match_any_sync(0xffffffffu, code);
            const int leader = __ffs(grp) - 1;
            int base = 0;
            if (ok && lane == leader) {
                const int cnt = __popc(grp);
                base = code < HIST_S ? offs_s[code] + atomicAdd(&scnt[code], cnt)
                                     : atomicAdd(sp.far_cur + (code - HIST_S), cnt);
            }
            base = __shfl_sync(0xffffffffu, base, leader);
            if (!ok) continue;
            const int d = base + __popc(grp & lt);
            if ((unsigned)d >= (unsigned)n_all) {
                ++n_bad;
                continue;
            }
            const int kb2 = kb_new[chunk_of(d, sp.div_m, sp.div_l)];
            pos[r].store(sp, nb, d);
            dvp_out[d] = dv[r] + (T)(kb - kb2) * dvk;
            fp_out[d] = f[r];
        }
    }
    if (n_bad) atomicAdd(&nbad_s, n_bad);
    __syncthreads();
    if (threadIdx.x == 0 && nbad_s) atomicOr(&ctl->err, ERR_CAPACITY);
}

// ---------------------------------------------------------------------------
// push + deposit + write back in place (one CTA per chunk)
// ---------------------------------------------------------------------------
// The deposit window is placed from the histogram of the chunk's current
// keys (cnt[hsel]: counted by the previous step, or, after a re-sort, the
// key ranges of the re-sorted chunks) and follows this step's drift column
// by column; every marker is pushed, deposited (runs of markers with the
// same footprint summed in registers first) and written back in place, and
// its new key is counted into cnt[1 - hsel] for the next step.  On a re-sort
// step the markers are read from the buffer k_rs1 has just written.
// FP64: one CTA per SM with the registers the push and deposit need (at two
// CTAs, 64 registers, it spills).
template <typename T, bool BATCH, bool PUSH>
__global__ void __launch_bounds__(PD_THREADS, sizeof(T) == 8 ? 1 : 2) k_pd1(const StepArgs* __restrict__ A0,
                                                       const BatchMap* __restrict__ bm)
{
    constexpr int mode = PUSH ? 1 : 0;
    extern __shared__ __align__(128) unsigned char smem[];
    int g = blockIdx.x;
    const StepArgs* __restrict__ A = A0;
    if constexpr (BATCH) A = batch_run(A0, bm, bm->pd_base, g);
    const int s = species_of_chunk(A, g);
    const SpDev& sp = A->sp[s];
    if (mode == 1 && !sp.mobile) return;
    Ctl* ctl = A->ctl;
    const bool push = mode == 1;
    const int hs = ctl->hsel[s];
    const int c = g - sp.chunk_base;
    const int nx = sp.nx, nv = sp.nvflat, W = sp.Wmax;
    const int cb = (push && ctl->sort_now[s]) ? 1 - ctl->cur[s] : ctl->cur[s];
    const int n_all = (int)sp.n;
    const int beg = c * sp.M, end = min((c + 1) * sp.M, n_all);
    const int kb = sp.KB[cb][c];
    const int kbase = kb - HIST_R;

    const size_t eb = ((size_t)nx * sizeof(T) + 15) & ~size_t(15);
    T* Es = reinterpret_cast<T*>(smem);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + eb);
    int* misc = reinterpret_cast<int*>(smem + eb + 16);   // [0] overflow runs, [2] row0
    int* scnt = reinterpret_cast<int*>(smem + eb + 32);   // next-step histogram
    int* hcur = scnt + HIST_S;                             // current-key histogram (window placement)
    int* shs = hcur + HIST_S;                              // per-column row shift (nx)
    unsigned char* winb = smem + eb + 32 + 2 * HIST_S * 4 + ((4 * nx + 15) & ~15);
    const int plane = win_plane(W, nx);
    const size_t win_bytes = (size_t)2 * sizeof(T) * plane;

    const T* Eg = (sizeof(T) == 4) ? reinterpret_cast<const T*>(A->fd.E32) : reinterpret_cast<const T*>(A->fd.E64);
    const bool use_bulk = push && ((nx * sizeof(T)) % 16 == 0);
    if (threadIdx.x == 0) {
        misc[0] = 0;
        if (use_bulk) {
            mbar_init(bar, 1);
            fence_mbar_init();
        }
    }
    for (int i = threadIdx.x; i < HIST_S; i += PD_THREADS) {
        scnt[i] = 0;
        hcur[i] = sp.cnt[hs][(size_t)c * HIST_S + i];
    }
    // window coordinate of a deposit at row j, column x: j - shs[x], which
    // removes this step's drift
    const int ssel = ctl->shsel[s];
    for (int i = threadIdx.x; i < nx; i += PD_THREADS) shs[i] = push ? sp.shift[ssel][i] : 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        const int r0 = best_window(hcur, kbase, W, nullptr);
        misc[2] = r0;
        sp.wrow0[c] = r0;
        if (use_bulk) {
            mbar_arrive_expect_tx(bar, (unsigned)(nx * sizeof(T)));
            bulk_g2s(Es, Eg, (unsigned)(nx * sizeof(T)), bar);
        }
    }
    {   // zero the window while the field is in flight
        float4* w4 = reinterpret_cast<float4*>(winb);
        const int n4 = (int)(win_bytes / 16);
        for (int i = threadIdx.x; i < n4; i += PD_THREADS) w4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (push && !use_bulk)
        for (int i = threadIdx.x; i < nx; i += PD_THREADS) Es[i] = Eg[i];
    // a first wait that gives up flags the timeout; the copy is drained and
    // the step goes on (every thread reaches the barrier below)
    if (use_bulk && !mbar_wait_or_drain(bar, 0, ctl->wait_limit, WAIT_LIMIT))
        if (threadIdx.x == 0) atomicOr(&ctl->err, ERR_TIMEOUT);
    __syncthreads();
    const int row0 = misc[2];

    T* win = reinterpret_cast<T*>(winb);
    // FP32: the reference plane, f of the previous reconstruction at every
    // window cell (grid row wr + row0 + shs[x] of column x; 0 off the grid)
    T* fref = win + 2 * plane;
    if constexpr (sizeof(T) == 4) {
        // eight rows' loads in flight per thread before their stores
        constexpr int RB = 8;
        const float* fprev = reinterpret_cast<const float*>(sp.fgrid);
        for (int x = threadIdx.x; x < nx; x += PD_THREADS) {
            const int j0x = row0 + shs[x];
            for (int wr0 = 0; wr0 < W; wr0 += RB) {
                float v[RB];
#pragma unroll
                for (int k = 0; k < RB; ++k) {
                    const int j = j0x + wr0 + k;
                    v[k] = (wr0 + k < W && (unsigned)j < (unsigned)nv) ? fprev[(size_t)j * nx + x] : 0.f;
                }
#pragma unroll
                for (int k = 0; k < RB; ++k)
                    if (wr0 + k < W) fref[(wr0 + k) * nx + x] = v[k];
            }
        }
        __syncthreads();
    }
    const T inv_dv = (T)sp.inv_dv[0];
    const T qm_dt = (T)sp.qm_dt;
    const T dt_dx = (T)sp.dt_dx;
    const T vref_dtdx = (T)((sp.vmin[0] + (double)kb * sp.dv[0]) * sp.dt_dx);
    // FP64: the displacement in 2^-52 cells (fixed-point positions, PosX)
    const double dt_dx52 = sp.dt_dx * PosX::ONE, vref_dtdx52 = (double)vref_dtdx * PosX::ONE;
    double* ovf_num = sp.ovf;
    double* ovf_den = sp.ovf + (size_t)nv * nx;
    int* ovf_tag = sp.ovf_tag;
    const int tag = (int)ctl->step + 1;
    T* dvp = reinterpret_cast<T*>(sp.mv[cb][0]);
    const T* fp = reinterpret_cast<const T*>(sp.mf[cb]);
    int* far_next = sp.far_cnt[1 - hs];
    unsigned n_over = 0;

    for (int base = beg; base < end; base += PD_THREADS * MPT) {
        const int g0 = base + threadIdx.x * MPT;
        const bool any = g0 < end;
        T dv8[MPT], f8[MPT];
        PosM<T> pos8[MPT];
        if (any) {
            loadg(dvp + g0, dv8);
            loadg(fp + g0, f8);
            if constexpr (sizeof(T) == 4) {
                int c8[MPT];
                float o8[MPT];
                loadg(reinterpret_cast<const int*>(sp.mx[cb]) + g0, c8);
                loadg(sp.moff[cb] + g0, o8);
#pragma unroll
                for (int m = 0; m < MPT; ++m) {
                    pos8[m].c = c8[m];
                    pos8[m].o = o8[m];
                }
            } else {
                long long x8[MPT];
                loadg(reinterpret_cast<const long long*>(sp.mx[cb]) + g0, x8);
#pragma unroll
                for (int m = 0; m < MPT; ++m) pos8[m].X = x8[m];
            }
        }
        Run<T> run;
        run.reset(0x7fffffff, 0);
        bool have = false;
        // one marker of the thread's group: push, footprint, run, key count
        auto one = [&](int m, bool okm) __attribute__((always_inline)) {
            int code = 0;
            if (okm) {
                PosM<T>& pos = pos8[m];
                T dv = dv8[m];
                const T fl = f8[m];
                if (push) {
                    int i0, ia, ib;
                    T w;
                    pos.cic(i0, w);
                    wrap_pair_in(i0, nx, ia, ib);
                    const T El = ((T)1 - w) * Es[ia] + w * Es[ib];
                    dv += qm_dt * El;
                    if constexpr (sizeof(T) == 8)
                        pos.drift_scaled(__fma_rn(dv, dt_dx52, vref_dtdx52), nx);   // in 2^-52 cells
                    else
                        pos.drift(vref_dtdx + dv * dt_dx, nx);
                    dv8[m] = dv;
                }
                // cloud-in-cell footprint of the new state (Eq. 4 weights)
                int i0;
                T wx;
                pos.cic(i0, wx);
                // the fused multiply-add of key_rel, so that the footprint row
                // is the key every other kernel computes from the stored value
                T t;
                if constexpr (sizeof(T) == 4)
                    t = __fmaf_rn(dv, inv_dv, -0.5f);
                else
                    t = __fma_rn(dv, inv_dv, -0.5);
                const T ft = floor(t);
                const int j0 = kb + (int)ft;
                code = rel_code(clampi(j0, 0, nv - 1), kbase);
                const T wv = t - ft;
                const bool first = !have || i0 != run.i0 || j0 != run.j0;
                if (first) {
                    if (have)
                        n_over += flush_run<T>(run, win, plane, row0, W, nx, nv, shs, fref, ovf_num, ovf_den, ovf_tag,
                                               tag)
                                      ? 1u
                                      : 0u;
                    run.reset(i0, j0);
                    have = true;
                }
                const T a[4] = {((T)1 - wx) * ((T)1 - wv), wx * ((T)1 - wv), ((T)1 - wx) * wv, wx * wv};
                run.add(a, fl, first);
            }
            // the new key counted for this chunk (next step's window)
            if (push) hist_add(scnt, far_next, code, okm);
        };
#pragma unroll
        for (int m = 0; m < MPT; ++m) one(m, g0 + m < end);
        if (have)
            n_over += flush_run<T>(run, win, plane, row0, W, nx, nv, shs, fref, ovf_num, ovf_den, ovf_tag, tag) ? 1u
                                                                                                                : 0u;
        if (!push) continue;
        // in place: the positions and velocities go back where they came from
        if (any) {
            storeg(dvp + g0, dv8);
            if constexpr (sizeof(T) == 4) {
                int c8[MPT];
                float o8[MPT];
#pragma unroll
                for (int m = 0; m < MPT; ++m) {
                    c8[m] = pos8[m].c;
                    o8[m] = pos8[m].o;
                }
                storeg(reinterpret_cast<int*>(sp.mx[cb]) + g0, c8);
                storeg(sp.moff[cb] + g0, o8);
            } else {
                long long x8[MPT];
#pragma unroll
                for (int m = 0; m < MPT; ++m) x8[m] = pos8[m].X;
                storeg(reinterpret_cast<long long*>(sp.mx[cb]) + g0, x8);
            }
        }
    }
    if (n_over) atomicAdd(&misc[0], (int)n_over);
    __syncthreads();
    if (push)
        for (int i = threadIdx.x; i < HIST_S; i += PD_THREADS) sp.cnt[1 - hs][(size_t)c * HIST_S + i] = scnt[i];
    // flush the window to this chunk's partial sums with one bulk copy
    if (threadIdx.x == 0) {
        fence_proxy_async_smem();
        unsigned char* dstp = reinterpret_cast<unsigned char*>(sp.partial) + (size_t)c * win_bytes;
        bulk_s2g(dstp, winb, (unsigned)win_bytes);
        bulk_commit();
        if (misc[0]) atomicAdd(&ctl->ovf_count[s], (unsigned long long)misc[0]);
        bulk_wait_all();
    }
}

// ---------------------------------------------------------------------------
// marker refinement: new markers traced back to the initial state (Sec. 2)
// ---------------------------------------------------------------------------
struct RefineArgs {
    int nx, nv, s, box[4], lat[2];
    double dx, L, vmin, dv, qm, dt, jitter;
    unsigned long long seed;
    int nhist;
    const double* Eh;    // [nhist][nx], E of the species' initial state first
    const avl_f0* f0;
    long long count;
};

// marker m of the box lattice (m = ((i - box0) rows + (j - box2)) ppc + a pv + b),
// jittered like the creation lattice, at the current time; then back along
// its characteristic by the inverse kick-drift step, x_n = x_{n+1} - v dt and
// v_n = v_{n+1} - (q/m) dt E^n(x_n), in FP64 without fused operations (the
// same sequence of roundings as a plain evaluation); f = f0 at the foot
__global__ void __launch_bounds__(256) k_refine1(RefineArgs R, double* __restrict__ xo, double* __restrict__ vo,
                                                 double* __restrict__ fo)
{
    const int ppc = R.lat[0] * R.lat[1];
    const int nrow = R.box[3] - R.box[2];
    for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < R.count;
         m += (long long)gridDim.x * blockDim.x) {
        const long long cell = m / ppc;
        const int sub = (int)(m - cell * ppc);
        const int i = R.box[0] + (int)(cell / nrow), j = R.box[2] + (int)(cell % nrow);
        const int a = sub / R.lat[1], b = sub - (sub / R.lat[1]) * R.lat[1];
        const double J0 = (jitter_u01(R.seed, R.s, m, 0) - 0.5) * R.jitter;
        const double J1 = (jitter_u01(R.seed, R.s, m, 1) - 0.5) * R.jitter;
        double x = ((double)i + ((double)a + 0.5 + J0) / R.lat[0]) * R.dx;
        double v = R.vmin + ((double)j + ((double)b + 0.5 + J1) / R.lat[1]) * R.dv;
        xo[m] = x;
        vo[m] = v;
        for (int n = R.nhist - 1; n >= 0; --n) {
            double xn = fmod(__dsub_rn(x, __dmul_rn(v, R.dt)), R.L);
            if (xn < 0.0) xn += R.L;
            if (xn >= R.L) xn -= R.L;
            x = xn;
            const double u = __dsub_rn(__ddiv_rn(x, R.dx), 0.5);
            const double fl = floor(u);
            const double w = __dsub_rn(u, fl);
            int ia, ib;
            wrap_pair((int)fl, R.nx, ia, ib);
            const double* E = R.Eh + (size_t)n * R.nx;
            const double El = __dadd_rn(__dmul_rn(__dsub_rn(1.0, w), E[ia]), __dmul_rn(w, E[ib]));
            v = __dsub_rn(v, __dmul_rn(__dmul_rn(R.qm, El), R.dt));
        }
        fo[m] = f0_value(R.f0, 1, R.L, x, &v);
    }
}

cudaError_t launch_refine1(const StepArgs& h, int s, const int box[4], const int lattice[2], const avl_f0* f0_dev,
                           unsigned long long seed, double jitter, double dt, int nhist, const double* Ehist,
                           long long count, double* x, double* v, double* f, cudaStream_t st)
{
    if (count == 0) return cudaSuccess;
    const SpDev& sp = h.sp[s];
    RefineArgs R;
    R.nx = sp.nx;
    R.nv = sp.nvflat;
    R.s = s;
    for (int k = 0; k < 4; ++k) R.box[k] = box[k];
    R.lat[0] = lattice[0];
    R.lat[1] = lattice[1];
    R.dx = sp.dx;
    R.L = sp.dx * sp.nx;
    R.vmin = sp.vmin[0];
    R.dv = sp.dv[0];
    R.qm = sp.qm;
    R.dt = dt;
    R.jitter = jitter;
    R.seed = seed;
    R.nhist = nhist;
    R.Eh = Ehist;
    R.f0 = f0_dev;
    R.count = count;
    const int blocks = (int)std::max<long long>(1, std::min<long long>((count + 255) / 256, 152ll * 8));
    k_refine1<<<blocks, 256, 0, st>>>(R, x, v, f);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// finalize: f = num / den (Eq. 4), charge per row group (Eq. 14), diagnostics
// ---------------------------------------------------------------------------
template <typename T>
struct CellSum;

// FP32: the window partials hold sum alpha (f_l - f_ref) and sum alpha
// (see Run<float>); they are summed over the chunks in float-float, the FP64
// overflow sums (absolute values) join as num - f_ref den, and
// f = f_ref + num / den is formed in float-float.
template <>
struct CellSum<float> {
    ff num{0.f, 0.f}, den{0.f, 0.f};
    __device__ __forceinline__ void add_partial(const float* p, int plane) { add_pair(p[0], p[plane]); }
    __device__ __forceinline__ void add_pair(float n, float d)
    {
        ff_add(num, n);
        ff_add(den, d);
    }
    __device__ __forceinline__ void add_ovf(double n, double d, float fr)
    {
        const double nd = n - (double)fr * d;
        ff_add(num, (float)nd);
        num.lo = __fadd_rn(num.lo, (float)(nd - (double)(float)nd));
        ff_add(den, (float)d);
        den.lo = __fadd_rn(den.lo, (float)(d - (double)(float)d));
    }
    // f = f_ref + num / den as float-float (fh, fl); den = 0 gives f = 0
    __device__ __forceinline__ void value(float fr, float& fh, float& fl, float& dsum) const
    {
        dsum = __fadd_rn(den.hi, den.lo);
        if (den.hi > 0.f) {
            const float q = __fdiv_rn(num.hi, den.hi);
            float r = fmaf(-q, den.hi, num.hi);
            r = __fadd_rn(r, __fsub_rn(num.lo, __fmul_rn(q, den.lo)));
            const float ql = __fdiv_rn(r, den.hi);
            float h = fr, l = 0.f;
            two_sum_add(h, l, q);
            fh = h;
            fl = __fadd_rn(l, ql);
        } else {
            fh = 0.f;
            fl = 0.f;
        }
    }
};

template <>
struct CellSum<double> {
    double num = 0.0, den = 0.0;
    __device__ __forceinline__ void add_partial(const double* p, int plane) { add_pair(p[0], p[plane]); }
    __device__ __forceinline__ void add_pair(double n, double d)
    {
        num += n;
        den += d;
    }
    __device__ __forceinline__ void add_ovf(double n, double d, double)
    {
        num += n;
        den += d;
    }
    __device__ __forceinline__ void value(double, double& fh, double& fl, double& dsum) const
    {
        dsum = den;
        fh = __double_as_longlong(den) > 0 ? div_nr(num, den) : 0.0;   // den >= 0 is a sum of weights
        fl = 0.0;
    }
};

constexpr int FIN_LIST = 256;  // chunks whose windows meet one finalize block's rows

template <typename T, bool BATCH>
__global__ void __launch_bounds__(FIN_THREADS, 4) k_fin1(const StepArgs* __restrict__ A0, int all_species,
                                                      const BatchMap* __restrict__ bm)
{
    constexpr int RL = FIN_THREADS / FIN_XB;   // row lanes
    __shared__ double col_red[RL][FIN_XB];
    __shared__ double red[3][FIN_THREADS / 32];
    __shared__ int clist[FIN_LIST];
    __shared__ int crow[FIN_LIST];
    __shared__ int ncl;
    int g = blockIdx.x;
    const StepArgs* __restrict__ A = A0;
    if constexpr (BATCH) A = batch_run(A0, bm, bm->fin_base, g);
    const int s = species_of_fin(A, g);
    const SpDev& sp = A->sp[s];
    if (!all_species && !sp.mobile) return;
    Ctl* ctl = A->ctl;
    const int blk = g - sp.fin_base;
    const int xb = blk % sp.nxb, rqi = blk / sp.nxb;
    const int nx = sp.nx, nv = sp.nvflat, W = sp.Wmax;
    const int col = threadIdx.x % FIN_XB, lr = threadIdx.x / FIN_XB;
    const int x = xb * FIN_XB + col;
    const bool xok = x < nx;
    const int j0 = rqi * sp.rq, j1 = min(nv, j0 + sp.rq);
    const int plane = win_plane(W, nx);
    const bool any_ovf = ctl->ovf_count[s] != 0;
    double* ovf_num = sp.ovf;
    double* ovf_den = sp.ovf + (size_t)nv * nx;
    const int* ovf_tag = sp.ovf_tag;
    const int tag = (int)ctl->step + 1;
    T* fg = reinterpret_cast<T*>(sp.fgrid);
    T* ng = reinterpret_cast<T*>(sp.ngrid);
    const T* part = reinterpret_cast<const T*>(sp.partial);
    constexpr int planes = 2;

    // chunks whose deposit windows meet rows [j0, j1), in chunk order (the
    // windows are stored shifted by shift[x] per column; all_species marks a
    // refresh, whose deposit used no shift)
    const bool shifted = !all_species && sp.mobile;
    const int ssel = ctl->shsel[s];
    const int smin = shifted ? ctl->shift_min[s][ssel] : 0;
    const int smax = shifted ? ctl->shift_max[s][ssel] : 0;
    const int shx = (shifted && xok) ? sp.shift[ssel][x] : 0;
    if (threadIdx.x == 0) ncl = 0;
    __syncthreads();
    for (int cc = threadIdx.x; cc < sp.nchunk; cc += FIN_THREADS) {
        const int r0 = sp.wrow0[cc];
        if (r0 + smin < j1 && r0 + W + smax > j0) {
            const int pos = atomicAdd(&ncl, 1);
            if (pos < FIN_LIST) {
                clist[pos] = cc;
                crow[pos] = r0;
            }
        }
    }
    __syncthreads();
    const int nlist = ncl;
    const bool use_list = nlist <= FIN_LIST;
    // the list ordered by first window row, ties by chunk (so that the sums
    // over windows keep one order whatever order the list was filled in); a
    // column walks only the windows that cover its rows
    __shared__ int slist[FIN_LIST], srow[FIN_LIST];
    if (use_list) {
        for (int t = threadIdx.x; t < nlist; t += FIN_THREADS) {
            const int r = crow[t], c = clist[t];
            int rank = 0;
            for (int q = 0; q < nlist; ++q) rank += (crow[q] < r || (crow[q] == r && clist[q] < c)) ? 1 : 0;
            slist[rank] = c;
            srow[rank] = r;
        }
        __syncthreads();
    }

    ColAcc<T> acc;
    if constexpr (sizeof(T) == 8) acc.logtab = A->fd.logtab;
    // overflow rows, f = num / den, f and n stored, charge and diagnostics
    // (FP32: f_ref = the cell's f of the previous reconstruction, read before
    // it is overwritten; the deposit kernel staged the same value)
    auto finish = [&](int j, CellSum<T>& cs) {
        const T fr = sizeof(T) == 4 ? fg[(size_t)j * nx + x] : (T)0;
        if (any_ovf && ovf_tag[j] == tag) {
            const size_t o = (size_t)j * nx + x;
            cs.add_ovf(ovf_num[o], ovf_den[o], fr);
            ovf_num[o] = 0.0;
            ovf_den[o] = 0.0;
        }
        T fh, fl, dsum;
        cs.value(fr, fh, fl, dsum);
        fg[(size_t)j * nx + x] = fh + fl;
        ng[(size_t)j * nx + x] = dsum;
        const T vj = (T)(sp.vmin[0] + (j + 0.5) * sp.dv[0]);
        acc.add(fh, fl, vj * vj);
    };
    if (xok && use_list) {
        // two rows at a time, the partials of their first WSLOT windows loaded
        // together (the loads of a row no longer wait for the previous row);
        // windows are added in list order, as one row at a time would
        constexpr int WSLOT = 3;
        const T* pcol = part + x;
        const size_t wstride = (size_t)planes * plane;
        int lo = 0;   // first listed window that can still reach the rows ahead
        for (int j = j0 + lr; j < j1; j += 2 * RL) {
            const int jb = j + RL;
            const bool two = jb < j1;
            const int ra = j - shx, rb = jb - shx;   // rows in window coordinates
            while (lo < nlist && srow[lo] + W <= ra) ++lo;
            int lob = lo;
            while (lob < nlist && srow[lob] + W <= rb) ++lob;
            T na[WSLOT], da[WSLOT], nb[WSLOT], db[WSLOT];
            bool oa[WSLOT], ob[WSLOT];
#pragma unroll
            for (int k = 0; k < WSLOT; ++k) {
                const int qa = lo + k, qb = lob + k;
                oa[k] = qa < nlist && srow[qa] <= ra;
                ob[k] = two && qb < nlist && srow[qb] <= rb;
                na[k] = da[k] = nb[k] = db[k] = (T)0;
                if (oa[k]) {
                    const T* pp = pcol + (size_t)slist[qa] * wstride + (size_t)(ra - srow[qa]) * nx;
                    na[k] = pp[0];
                    da[k] = pp[plane];
                }
                if (ob[k]) {
                    const T* pp = pcol + (size_t)slist[qb] * wstride + (size_t)(rb - srow[qb]) * nx;
                    nb[k] = pp[0];
                    db[k] = pp[plane];
                }
            }
            CellSum<T> ca, cb;
#pragma unroll
            for (int k = 0; k < WSLOT; ++k)
                if (oa[k]) ca.add_pair(na[k], da[k]);
            for (int q = lo + WSLOT; q < nlist && srow[q] <= ra; ++q)
                ca.add_partial(pcol + (size_t)slist[q] * wstride + (size_t)(ra - srow[q]) * nx, plane);
            finish(j, ca);
            if (two) {
#pragma unroll
                for (int k = 0; k < WSLOT; ++k)
                    if (ob[k]) cb.add_pair(nb[k], db[k]);
                for (int q = lob + WSLOT; q < nlist && srow[q] <= rb; ++q)
                    cb.add_partial(pcol + (size_t)slist[q] * wstride + (size_t)(rb - srow[q]) * nx, plane);
                finish(jb, cb);
            }
            lo = lob;
        }
    } else if (xok) {
        // more windows meet these rows than the list holds: scan every chunk
        for (int j = j0 + lr; j < j1; j += RL) {
            CellSum<T> cs;
            for (int cc = 0; cc < sp.nchunk; ++cc) {
                const int wr = j - shx - sp.wrow0[cc];
                if (wr >= 0 && wr < W) cs.add_partial(part + (size_t)cc * planes * plane + (size_t)wr * nx + x, plane);
            }
            finish(j, cs);
        }
    }
    // charge of this species per column, summed over the row lanes in order
    col_red[lr][col] = acc.r();
    __syncthreads();
    if (lr == 0 && xok) {
        double r = 0.0;
        for (int k = 0; k < RL; ++k) r += col_red[k][col];
        sp.rho_part[(size_t)rqi * nx + x] = sp.q * sp.dv[0] * r;
    }
    // diagnostics of the block
    double dN = acc.r(), dW = acc.wk(), dS = acc.s();
    for (int o = 16; o > 0; o >>= 1) {
        dN += __shfl_down_sync(0xffffffffu, dN, o);
        dW += __shfl_down_sync(0xffffffffu, dW, o);
        dS += __shfl_down_sync(0xffffffffu, dS, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[0][warp] = dN;
        red[1][warp] = dW;
        red[2][warp] = dS;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, bb = 0, cc = 0;
        for (int w = 0; w < FIN_THREADS / 32; ++w) {
            a += red[0][w];
            bb += red[1][w];
            cc += red[2][w];
        }
        const double cell = sp.dx * sp.dv[0];
        sp.dpart[(size_t)blk * 4 + 0] = a * cell;
        sp.dpart[(size_t)blk * 4 + 1] = 0.5 * sp.m * bb * cell;
        sp.dpart[(size_t)blk * 4 + 2] = cc * cell;
        sp.dpart[(size_t)blk * 4 + 3] = 0.0;
    }
}

// ---------------------------------------------------------------------------
// marker sources for creation: the jittered lattice and caller arrays
// ---------------------------------------------------------------------------
struct MarkerIn {
    double xi;   // position in cells
    double v;
    double f;
    bool ok;
};

// lattice marker number k in generation order (velocity row j slowest, then
// cell i, then sub-point p), which is nearly sorted by key; the jitter stream
// uses the row-major marker number (cell * ppc + p)
struct LatticeSrc {
    const avl_f0* f0;
    unsigned long long seed;
    double jitter;
    int s, px, pv;
    __device__ MarkerIn get(const SpDev& sp, long long k) const
    {
        const int ppc = px * pv;
        const long long per_row = (long long)sp.nx * ppc;
        const int j = (int)(k / per_row);
        const long long rem = k - (long long)j * per_row;
        const int i = (int)(rem / ppc);
        const int p = (int)(rem - (long long)i * ppc);
        const int a = p / pv, bv = p - a * pv;
        const long long m = ((long long)i * sp.nvflat + j) * ppc + p;
        const double J0 = (jitter_u01(seed, s, m, 0) - 0.5) * jitter;
        const double J1 = (jitter_u01(seed, s, m, 1) - 0.5) * jitter;
        MarkerIn r;
        r.xi = (double)i + ((double)a + 0.5 + J0) / px;
        const double v[3] = {sp.vmin[0] + ((double)j + ((double)bv + 0.5 + J1) / pv) * sp.dv[0], 0.0, 0.0};
        r.v = v[0];
        r.f = f0_value(f0, 1, sp.nx * sp.dx, r.xi * sp.dx, v);
        r.ok = true;
        return r;
    }
};

struct ArraySrc {
    const double* x;
    const double* v;
    const double* f;
    __device__ MarkerIn get(const SpDev& sp, long long k) const
    {
        MarkerIn r;
        const double L = sp.nx * sp.dx;
        const double xv = x[k];
        r.v = v[k];
        r.f = f[k];
        r.ok = (xv >= 0.0 && xv < L) && isfinite(r.v) && isfinite(r.f);
        r.xi = r.ok ? xv / sp.dx : 0.0;
        if (!r.ok) {
            r.v = sp.vmin[0];
            r.f = 0.0;
        }
        return r;
    }
};

// key histogram of a source chunk; its reference key = key of its first marker
template <typename Src>
__global__ void __launch_bounds__(CNT_THREADS) k_src_count(const StepArgs* __restrict__ A, int s, Src src,
                                                          unsigned long long* bad)
{
    __shared__ int hist[HIST_S];
    __shared__ int kref_s;
    const SpDev& sp = A->sp[s];
    const int c = blockIdx.x;
    const long long beg = (long long)c * sp.M, end = min((long long)(c + 1) * sp.M, sp.n);
    const int nv = sp.nvflat;
    for (int i = threadIdx.x; i < HIST_S; i += CNT_THREADS) hist[i] = 0;
    if (threadIdx.x == 0) {
        kref_s = key_abs(src.get(sp, beg).v, sp.vmin[0], sp.inv_dv[0], nv);
        sp.kref_tmp[c] = kref_s;
    }
    __syncthreads();
    const int kbase = kref_s - HIST_R;
    unsigned nbad = 0;
    for (long long b0 = beg; b0 < end; b0 += CNT_THREADS) {
        const long long k = b0 + threadIdx.x;
        const bool ok = k < end;
        int code = 0;
        if (ok) {
            const MarkerIn mk = src.get(sp, k);
            if (!mk.ok) nbad++;
            code = rel_code(key_abs(mk.v, sp.vmin[0], sp.inv_dv[0], nv), kbase);
        }
        hist_add(hist, sp.far_cnt[0], code, ok);
    }
    if (nbad && bad) atomicAdd(bad, (unsigned long long)nbad);
    __syncthreads();
    for (int i = threadIdx.x; i < HIST_S; i += CNT_THREADS) sp.cnt[0][(size_t)c * HIST_S + i] = hist[i];
}

__global__ void __launch_bounds__(512) k_src_scan(const StepArgs* __restrict__ A, int s)
{
    const SpDev& sp = A->sp[s];
    // source chunk references are not ordered: every chunk is visited per key;
    // the new layout goes to buffer 0
    scan_layout(sp, sp.kref_tmp, sp.cnt[0], sp.far_cnt[0], false, sp.KB[0]);
}

template <typename T, typename Src>
__global__ void __launch_bounds__(PD_THREADS) k_src_scatter(const StepArgs* __restrict__ A, int s, Src src)
{
    __shared__ int scnt[HIST_S];
    __shared__ unsigned nbad_s;
    const SpDev& sp = A->sp[s];
    const int c = blockIdx.x;
    const int n_all = (int)sp.n;
    const int beg = c * sp.M, end = min((c + 1) * sp.M, n_all);
    const int nv = sp.nvflat;
    const int kbase = sp.kref_tmp[c] - HIST_R;
    for (int i = threadIdx.x; i < HIST_S; i += PD_THREADS) scnt[i] = 0;
    if (threadIdx.x == 0) nbad_s = 0;
    __syncthreads();
    const int* offs = sp.offs + (size_t)c * HIST_S;
    for (int base = beg; base < end; base += PD_THREADS * MPT) {
        const int g0 = base + threadIdx.x * MPT;
        int code[MPT], dst[MPT];
#pragma unroll
        for (int m = 0; m < MPT; ++m) {
            const int k = g0 + m;
            code[m] = k < end ? rel_code(key_abs(src.get(sp, k).v, sp.vmin[0], sp.inv_dv[0], nv), kbase) : -1;
        }
        assign_slots(code, scnt, offs, sp.far_cur, dst);
#pragma unroll
        for (int m = 0; m < MPT; ++m) {
            const int k = g0 + m;
            if (k < end) {
                const MarkerIn mk = src.get(sp, k);
                const int d = dst[m];
                if ((unsigned)d < (unsigned)n_all) {
                    const int c2 = chunk_of(d, sp.div_m, sp.div_l);
                    const PosM<T> p = posm_from_cells<T>(mk.xi, sp.nx);
                    p.store(sp, 0, d);
                    const double vref = sp.vmin[0] + (double)sp.KB[0][c2] * sp.dv[0];
                    reinterpret_cast<T*>(sp.mv[0][0])[d] = (T)(mk.v - vref);
                    reinterpret_cast<T*>(sp.mf[0])[d] = (T)mk.f;
                } else {
                    atomicAdd(&nbad_s, 1u);
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && nbad_s) atomicOr(&A->ctl->err, ERR_CAPACITY);
}

template <typename T>
__global__ void k_get1(const StepArgs* __restrict__ A, int s, double* __restrict__ x, double* __restrict__ v,
                       double* __restrict__ f)
{
    const SpDev& sp = A->sp[s];
    const int c = blockIdx.x;
    const int cb = A->ctl->cur[s];
    const int beg = c * sp.M, end = (int)min((long long)(c + 1) * sp.M, sp.n);
    const double vref = sp.vmin[0] + (double)sp.KB[cb][c] * sp.dv[0];
    for (int k = beg + threadIdx.x; k < end; k += blockDim.x) {
        PosM<T> pos;
        pos.load(sp, cb, k);
        if (x) x[k] = pos.cells() * sp.dx;
        if (v) v[k] = vref + (double)reinterpret_cast<const T*>(sp.mv[cb][0])[k];
        if (f) f[k] = (double)reinterpret_cast<const T*>(sp.mf[cb])[k];
    }
}

template <typename T>
__global__ void k_getf(const T* __restrict__ fg, const T* __restrict__ ng, int nx, int nvflat,
                       double* __restrict__ f, double* __restrict__ n)
{
    // internal [v][x] -> caller [x][v]
    __shared__ double tile[2][32][33];
    const int xb = blockIdx.x * 32, vb = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int vj = vb + r, xi = xb + threadIdx.x;
        if (vj < nvflat && xi < nx) {
            tile[0][r][threadIdx.x] = (double)fg[(size_t)vj * nx + xi];
            if (n) tile[1][r][threadIdx.x] = (double)ng[(size_t)vj * nx + xi];
        }
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int xi = xb + r, vj = vb + threadIdx.x;
        if (vj < nvflat && xi < nx) {
            f[(size_t)xi * nvflat + vj] = tile[0][threadIdx.x][r];
            if (n) n[(size_t)xi * nvflat + vj] = tile[1][threadIdx.x][r];
        }
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_pd1_batch(int prec, const BatchMap* bm, int blocks, int smem, int mode, cudaStream_t st)
{
    if (blocks == 0) return cudaSuccess;
    if (prec == AVL_FP32) {
        if (mode == 1)
            k_pd1<float, true, true><<<blocks, PD_THREADS, smem, st>>>(nullptr, bm);
        else
            k_pd1<float, true, false><<<blocks, PD_THREADS, smem, st>>>(nullptr, bm);
    } else {
        if (mode == 1)
            k_pd1<double, true, true><<<blocks, PD_THREADS, smem, st>>>(nullptr, bm);
        else
            k_pd1<double, true, false><<<blocks, PD_THREADS, smem, st>>>(nullptr, bm);
    }
    return cudaGetLastError();
}

cudaError_t launch_rs1_batch(int prec, const BatchMap* bm, int blocks, cudaStream_t st)
{
    if (blocks == 0) return cudaSuccess;
    if (prec == AVL_FP32)
        k_rs1<float, true><<<blocks, PD_THREADS, 0, st>>>(nullptr, bm);
    else
        k_rs1<double, true><<<blocks, PD_THREADS, 0, st>>>(nullptr, bm);
    return cudaGetLastError();
}

cudaError_t launch_fin1_batch(int prec, const BatchMap* bm, int blocks, int all_species, cudaStream_t st)
{
    if (blocks == 0) return cudaSuccess;
    if (prec == AVL_FP32)
        k_fin1<float, true><<<blocks, FIN_THREADS, 0, st>>>(nullptr, all_species, bm);
    else
        k_fin1<double, true><<<blocks, FIN_THREADS, 0, st>>>(nullptr, all_species, bm);
    return cudaGetLastError();
}

static int max_pd_smem(const StepArgs& h)
{
    size_t m = 0;
    for (int s = 0; s < h.ns; ++s)
        if (h.sp[s].nchunk) m = std::max(m, pd1_smem_bytes(h.sp[s], h.prec));
    return (int)std::max<size_t>(m, 1024);
}

int pd1_smem_needed(const StepArgs& h) { return max_pd_smem(h); }

// dynamic shared-memory limit of the deposit kernel, set whenever the chunk
// layout changes (outside any stream capture)
template <typename T>
static cudaError_t set_pd1_limit_t(int smem)
{
    cudaError_t e;
    if ((e = raise_smem_limit(k_pd1<T, false, false>, smem))) return e;
    if ((e = raise_smem_limit(k_pd1<T, false, true>, smem))) return e;
    if ((e = raise_smem_limit(k_pd1<T, true, false>, smem))) return e;
    return raise_smem_limit(k_pd1<T, true, true>, smem);
}

static cudaError_t set_pd1_limit(int prec, int smem)
{
    return prec == AVL_FP32 ? set_pd1_limit_t<float>(smem) : set_pd1_limit_t<double>(smem);
}

cudaError_t configure_vhs1(const StepArgs& h) { return set_pd1_limit(h.prec, max_pd_smem(h)); }

cudaError_t configure_batch1(int prec, int pd_smem, int field_smem)
{
    cudaError_t e = set_pd1_limit(prec, pd_smem);
    if (e) return e;
    return configure_field_bytes(field_smem);
}

cudaError_t launch_count1(const StepArgs& h, const StepArgs* d, cudaStream_t st)
{
    if (h.nchunk_total == 0) return cudaSuccess;
    if (h.prec == AVL_FP32)
        k_count1<float><<<h.nchunk_total, CNT_THREADS, 0, st>>>(d);
    else
        k_count1<double><<<h.nchunk_total, CNT_THREADS, 0, st>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_pd1(const StepArgs& h, const StepArgs* d, int mode, cudaStream_t st)
{
    if (h.nchunk_total == 0) return cudaSuccess;
    const int smem = max_pd_smem(h);
    if (h.prec == AVL_FP32) {
        if (mode == 1)
            k_pd1<float, false, true><<<h.nchunk_total, PD_THREADS, smem, st>>>(d, nullptr);
        else
            k_pd1<float, false, false><<<h.nchunk_total, PD_THREADS, smem, st>>>(d, nullptr);
    } else {
        if (mode == 1)
            k_pd1<double, false, true><<<h.nchunk_total, PD_THREADS, smem, st>>>(d, nullptr);
        else
            k_pd1<double, false, false><<<h.nchunk_total, PD_THREADS, smem, st>>>(d, nullptr);
    }
    return cudaGetLastError();
}

cudaError_t launch_rs1(const StepArgs& h, const StepArgs* d, cudaStream_t st)
{
    if (h.nchunk_total == 0) return cudaSuccess;
    if (h.prec == AVL_FP32)
        k_rs1<float, false><<<h.nchunk_total, PD_THREADS, 0, st>>>(d, nullptr);
    else
        k_rs1<double, false><<<h.nchunk_total, PD_THREADS, 0, st>>>(d, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_fin1(const StepArgs& h, const StepArgs* d, int all_species, cudaStream_t st)
{
    if (h.prec == AVL_FP32)
        k_fin1<float, false><<<h.nfin_total, FIN_THREADS, 0, st>>>(d, all_species, nullptr);
    else
        k_fin1<double, false><<<h.nfin_total, FIN_THREADS, 0, st>>>(d, all_species, nullptr);
    return cudaGetLastError();
}

// source -> sorted layout in buffer 0 of species s (uses cnt[0], far_cnt[0],
// which the caller zeroes first, as scratch)
template <typename Src>
static cudaError_t source_to_layout(const StepArgs& h, const StepArgs* d, int s, Src src, unsigned long long* bad,
                                    cudaStream_t st)
{
    const SpDev& sp = h.sp[s];
    k_src_count<Src><<<sp.nchunk, CNT_THREADS, 0, st>>>(d, s, src, bad);
    k_src_scan<<<1, 512, 0, st>>>(d, s);
    if (h.prec == AVL_FP32)
        k_src_scatter<float, Src><<<sp.nchunk, PD_THREADS, 0, st>>>(d, s, src);
    else
        k_src_scatter<double, Src><<<sp.nchunk, PD_THREADS, 0, st>>>(d, s, src);
    return cudaGetLastError();
}

cudaError_t launch_init1(const StepArgs& h, const StepArgs* d, int s, const int lattice[4], const avl_f0* f0_dev,
                         unsigned long long seed, double jitter, cudaStream_t st)
{
    const LatticeSrc src{f0_dev, seed, jitter, s, lattice[0], lattice[1]};
    return source_to_layout(h, d, s, src, nullptr, st);
}

cudaError_t launch_set1(const StepArgs& h, const StepArgs* d, int s, long long, const double* x, const double* v,
                        const double* f, unsigned long long* bad, cudaStream_t st)
{
    const ArraySrc src{x, v, f};
    return source_to_layout(h, d, s, src, bad, st);
}

cudaError_t launch_get1(const StepArgs& h, const StepArgs* d, int s, double* x, double* v, double* f,
                        cudaStream_t st)
{
    if (h.sp[s].nchunk == 0) return cudaSuccess;
    if (h.prec == AVL_FP32)
        k_get1<float><<<h.sp[s].nchunk, 256, 0, st>>>(d, s, x, v, f);
    else
        k_get1<double><<<h.sp[s].nchunk, 256, 0, st>>>(d, s, x, v, f);
    return cudaGetLastError();
}

cudaError_t launch_getf(const StepArgs& h, int s, double* f, double* n, cudaStream_t st)
{
    const SpDev& sp = h.sp[s];
    dim3 grid((sp.nx + 31) / 32, (sp.nvflat + 31) / 32);
    dim3 block(32, 8);
    if (h.prec == AVL_FP32)
        k_getf<float><<<grid, block, 0, st>>>(reinterpret_cast<const float*>(sp.fgrid),
                                              reinterpret_cast<const float*>(sp.ngrid), sp.nx, sp.nvflat, f, n);
    else
        k_getf<double><<<grid, block, 0, st>>>(reinterpret_cast<const double*>(sp.fgrid),
                                               reinterpret_cast<const double*>(sp.ngrid), sp.nx, sp.nvflat, f, n);
    return cudaGetLastError();
}

}  // namespace avl
