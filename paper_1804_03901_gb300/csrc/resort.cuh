// resort.cuh -- device helpers for the velocity-row layout of the markers:
// key codes, deposit-window placement from a chunk's key histogram, and the
// scan that turns per-chunk key counts into the slots of a re-sorted layout.
// Included by the push kernel (k_vhs1.cu) and by the field kernel
// (k_field.cu), whose spare cluster CTA runs the scan.
#pragma once
#include "avl_internal.cuh"

namespace avl {

// key code used by the histograms and slot assignment: [0, HIST_S) inside
// the chunk's histogram window (keys kbase .. kbase + HIST_S - 1), HIST_S +
// key for keys outside it ("far" keys)
__device__ __forceinline__ int rel_code(int key, int kbase)
{
    const int r = key - kbase;
    return (r >= 0 && r < HIST_S) ? r : HIST_S + key;
}

// Deposit window of a chunk from the histogram of its markers' keys (the
// dual rows of the current state): the placement of wk consecutive keys that
// holds the most markers.  Returns the first window row (the window spans
// Wmax rows: HALO rows of drift below, wk key rows, HALO + 1 rows above).
__device__ __forceinline__ int best_window(const int* hist, int kbase, int wmax, int* covered)
{
    const int wk = max(1, min(HIST_S, wmax - 2 * HALO - 1));
    int sum = 0;
    for (int r = 0; r < wk; ++r) sum += hist[r];
    int best = sum, bestr = 0;
    for (int r = 1; r + wk <= HIST_S; ++r) {
        sum += hist[r + wk - 1] - hist[r - 1];
        if (sum > best) {
            best = sum;
            bestr = r;
        }
    }
    if (covered) *covered = best;
    return kbase + bestr - HALO;
}

// chunks whose histogram window (kref[c] - HIST_R + [0, HIST_S)) contains key
// k: a contiguous range because kref is non-decreasing over chunks
__device__ __forceinline__ void chunk_range(const int* kref, int nch, int k, bool sorted, int& c0, int& c1)
{
    c0 = 0;
    c1 = nch;
    if (!sorted) return;
    int lo = 0, hi = nch;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (kref[mid] - HIST_R > k - HIST_S) hi = mid; else lo = mid + 1;
    }
    c0 = lo;
    hi = nch;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (kref[mid] - HIST_R > k) hi = mid; else lo = mid + 1;
    }
    c1 = lo;
}

// Slots of the re-sorted layout from the key counts cnt[c][r] of every chunk c
// (keys kref[c] - HIST_R + r) and far_cnt[k] of the far keys.  Writes
// base_new (first slot of each key), offs[c][r] (first slot of chunk c's
// markers of that key; chunks in order), far_cur[k] (first slot of the far
// markers of key k) and, if kb_new is given, the reference key of every
// chunk of the new layout (the key of its first slot).  kref is staged in
// shared memory when it fits; base_s, if given, is block shared memory of
// nvflat + 1 ints where the scan runs (and keeps base_new for the caller).
// Called by a whole block.
static __device__ void scan_layout(const SpDev& sp, const int* __restrict__ kref_g, const int* __restrict__ cnt,
                            const int* __restrict__ far_cnt, bool sorted, int* kb_new, int* base_s = nullptr)
{
    const int nv = sp.nvflat, nch = sp.nchunk;
    __shared__ int warp_sums[32];
    __shared__ int carry;
    __shared__ int kref_s[1024];
    const int* kref = kref_g;
    if (nch <= 1024) {
        for (int c = threadIdx.x; c < nch; c += blockDim.x) kref_s[c] = kref_g[c];
        kref = kref_s;
    }
    int* base = base_s ? base_s : sp.base_new;
    __syncthreads();
    // (a) totals per key
    for (int k = threadIdx.x; k < nv; k += blockDim.x) {
        int tot = far_cnt[k];
        int c0, c1;
        chunk_range(kref, nch, k, sorted, c0, c1);
#pragma unroll 4
        for (int c = c0; c < c1; ++c) {
            const int r = k - (kref[c] - HIST_R);
            if (r >= 0 && r < HIST_S) tot += cnt[(size_t)c * HIST_S + r];
        }
        base[k] = tot;
    }
    __syncthreads();
    // (b) exclusive scan over keys
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int b0 = 0; b0 < nv; b0 += blockDim.x) {
        const int i = b0 + threadIdx.x;
        const int v = i < nv ? base[i] : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = lane < nw ? warp_sums[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            warp_sums[lane] = w;
        }
        __syncthreads();
        const int incl = x + (warp > 0 ? warp_sums[warp - 1] : 0) + carry;
        if (i < nv) base[i] = incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) base[nv] = carry;
    __syncthreads();
    if (base_s)
        for (int k = threadIdx.x; k <= nv; k += blockDim.x) sp.base_new[k] = base_s[k];
    // (c) first slot of every (chunk, key), then of the far markers of each key
    for (int k = threadIdx.x; k < nv; k += blockDim.x) {
        int run = base[k];
        int c0, c1;
        chunk_range(kref, nch, k, sorted, c0, c1);
#pragma unroll 4
        for (int c = c0; c < c1; ++c) {
            const int r = k - (kref[c] - HIST_R);
            if (r >= 0 && r < HIST_S) {
                sp.offs[(size_t)c * HIST_S + r] = run;
                run += cnt[(size_t)c * HIST_S + r];
            }
        }
        sp.far_cur[k] = run;
    }
    __syncthreads();
    // (d) reference key of every chunk of the new layout
    if (kb_new) {
        for (int c = threadIdx.x; c < nch; c += blockDim.x) {
            const int p = c * sp.M;
            int lo = 0, hi = nv;   // largest k with base_new[k] <= p
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (base[mid] <= p) lo = mid; else hi = mid;
            }
            kb_new[c] = lo;
        }
    }
    __syncthreads();
}

// Key histograms of the chunks of a layout sorted by key, from the first
// slot of every key (base: base_new as scan_layout left it, in global or
// shared memory): cnt_out[c][r] = the slots of chunk c ([c M, (c + 1) M))
// that hold key kb_new[c] - HIST_R + r.  Called by a whole block after
// scan_layout.
static __device__ void sorted_chunk_hist(const SpDev& sp, const int* __restrict__ kb_new, int* __restrict__ cnt_out,
                                         const int* base)
{
    const int nv = sp.nvflat;
    const long long total = (long long)sp.nchunk * HIST_S;
    for (long long i = threadIdx.x; i < total; i += blockDim.x) {
        const int c = (int)(i / HIST_S), r = (int)(i % HIST_S);
        const int k = kb_new[c] - HIST_R + r;
        int n = 0;
        if (k >= 0 && k < nv) {
            const long long lo = max((long long)base[k], (long long)c * sp.M);
            const long long hi = min((long long)base[k + 1], min((long long)(c + 1) * sp.M, sp.n));
            n = hi > lo ? (int)(hi - lo) : 0;
        }
        cnt_out[i] = n;
    }
    __syncthreads();
}

}  // namespace avl
