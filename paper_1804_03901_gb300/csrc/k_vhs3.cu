// k_vhs3.cu -- 1d3v kernels of the Vlasov-Hybrid time step (Fig. 2; Sec. 2
// with three velocity dimensions).
//
// Without a magnetic field the field changes v_x only and v_y, v_z ride
// along unchanged.  Layout: markers sorted by pencil (the dual rows of v_y and
// v_z, fixed for the life of a marker) and inside a pencil by key (dual row
// of v_x + 1).  One CTA owns one pencil and walks its keys in order; per
// segment (the markers stored under one key):
//   push    gather E (cloud-in-cell, Sec. 2), v_x += (q/m) E dt, x += v_x dt,
//           written back in place
//   sort    the markers whose new key is still the segment's key ("stays")
//           are counting-sorted by their x dual cell in shared memory
//   gather  one thread per x column adds the 16 cloud-in-cell weights (Eq. 4
//           numerator alpha f and denominator alpha) of the markers of its
//           two dual cells into registers: rows j, j+1 of v_x times the
//           pencil's four (v_y, v_z) cells -- no atomics.  FP64: the columns
//           are counting-sorted by their pair counts, their sums kept in
//           shared-memory row planes, and each of 128 lanes walks a light
//           and a heavy column in one loop, so that a warp's lanes do nearly
//           equal work (an FP64 warp instruction costs its SM sub-partition
//           the same whatever its active lanes); the weights of a marker's
//           (v_y, v_z) cells are stored beside it
//   flush   a finished v_x row is added into the global accumulators; each
//           cell receives the sums of the four pencils that reach it
// Markers whose key moved since the last re-sort deposit their 16
// contributions through global reductions, one thread per contribution;
// their counts decide the next re-sort (k_sort3, per pencil, into the other
// buffer).  k_fin3 forms f = num / den, the moment (Eq. 14) and the
// diagnostics (Sec. 3.4.1) and clears the other accumulator.
//
// With a static background magnetic field (Sec. 3.2: the Boris push of the
// 1d3v version) every velocity component turns, so a marker's pencil changes
// from step to step.  The step is then: Boris push in place with the count of
// every marker's new (pencil, key) bucket (k_bpush3), a global counting sort
// into the other buffer (k_src3_tsum, k_src3_scan, k_rs3_scatter,
// k_src3_flip), and the pencil deposit above without a push (k_pd3 mode 2),
// in which no marker is off its segment.
#include <math.h>

#include <algorithm>

#include "avl_internal.cuh"
#include "common.cuh"
#include "ptx.cuh"

namespace avl {

// position type of the 1d3v kernels (common.cuh): FP32 int cell + FP32
// offset, FP64 PosX
template <typename T>
using Pos3 = PosM<T>;

template <typename T>
__device__ __forceinline__ Pos3<T> pos3_from_cells(double xi, int nx)
{
    return posm_from_cells<T>(xi, nx);
}

template <typename T>
struct Cfg3;
template <>
struct Cfg3<float> {
    static constexpr int MPT = 2;   // markers per thread and chunk
};
template <>
struct Cfg3<double> {
    static constexpr int MPT = 2;
};

__device__ __forceinline__ int species_of_pen(const StepArgs* A, int g)
{
    int s = 0;
    while (s + 1 < A->ns && g >= A->sp[s + 1].pen_base) ++s;
    return s;
}

__device__ __forceinline__ int species_of_fin3(const StepArgs* A, int g)
{
    int s = 0;
    while (s + 1 < A->ns && g >= A->sp[s + 1].fin_base) ++s;
    return s;
}

// Dual row of a velocity component on a grid of n cells: t = v a + b with
// a = 1/dv and b = -vmin/dv - 1/2 (the cloud-in-cell rule of Fig. 1 on a
// cell-centred grid).  Returns floor(t) limited to [-2, n] (-2 and n: the
// footprint misses the grid) and the weight w = t - floor(t) of row j + 1.
// One explicit fused multiply-add, so that every kernel finds the same row.
__device__ __forceinline__ int dual3(float v, float a, float b, int n, float& w)
{
    const float t = __fmaf_rn(v, a, b);
    if (!(t > -2.0f && t < (float)n)) {
        w = 0.0f;
        return t > 0.0f ? n : -2;
    }
    const float fl = floorf(t);
    w = t - fl;
    return (int)fl;
}
// FP64: a and b come scaled by 2^52 (dual_coef), so that t 2^52 rounds to a
// 64-bit count of 2^-52 rows in one saturating conversion (NaN gives 0);
// the row is its high bits and the weight its low 52 bits, read as the
// mantissa of 1 + w: the FP64 pipe (the kernel's limit) sees three
// operations, the range test is in integers
__device__ __forceinline__ int dual3(double v, double a52, double b52, int n, double& w)
{
    const long long t = __double2ll_rn(__fma_rn(v, a52, b52));
    const int fl = (int)(t >> 52);
    if (fl < -2 || fl >= n) {
        w = 0.0;
        return fl < 0 ? -2 : n;
    }
    w = __longlong_as_double(0x3FF0000000000000ll | (t & 0x000FFFFFFFFFFFFFll)) - 1.0;
    return fl;
}

// coefficients a, b of dual3 for dimension d of a species, in storage
// precision (FP64: times 2^52)
template <typename T>
__device__ __forceinline__ void dual_coef(const SpDev& sp, int d, T& a, T& b)
{
    const double s = sizeof(T) == 8 ? 4503599627370496.0 : 1.0;
    a = (T)(sp.inv_dv[d] * s);
    b = (T)((-sp.vmin[d] * sp.inv_dv[d] - 0.5) * s);
}

template <typename T>
struct VCoef {
    T a[3], b[3];
    int n[3];
    __device__ __forceinline__ void init(const SpDev& sp)
    {
        for (int d = 0; d < 3; ++d) {
            dual_coef<T>(sp, d, a[d], b[d]);
            n[d] = sp.nv[d];
        }
    }
};

__device__ __forceinline__ int key_of(int j, int n) { return clampi(j, -1, n - 1) + 1; }

// warp-aggregated slot: lanes with equal keys take consecutive slots of
// cur[key] (one atomic per distinct key in the warp); lanes with ok = false
// take part but get no slot
__device__ __forceinline__ int warp_slot(int* cur, int key, bool ok)
{
    const int kk = ok ? key : -1;
    const unsigned grp = __match_any_sync(0xffffffffu, kk);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(grp) - 1;
    int base = 0;
    if (ok && lane == leader) base = atomicAdd(&cur[key], __popc(grp));
    base = __shfl_sync(0xffffffffu, base, leader);
    return base + __popc(grp & ((1u << lane) - 1u));
}

// exclusive scan of in[0, n) into out[0, n], out[n] = total, by a block of
// P3_THREADS threads; each thread takes `items` consecutive entries
// (items * P3_THREADS >= n); in may alias out
__device__ void block_exscan(const int* in, int* out, int n, int items, int* wsum)
{
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int i0 = t * items;
    int loc = 0;
    for (int i = 0; i < items; ++i)
        if (i0 + i < n) loc += in[i0 + i];
    int x = loc;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < P3_THREADS / 32 ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < P3_THREADS / 32) wsum[lane] = w;
    }
    __syncthreads();
    int run = x - loc + (warp > 0 ? wsum[warp - 1] : 0);
    for (int i = 0; i < items; ++i)
        if (i0 + i < n) {
            const int v = in[i0 + i];
            out[i0 + i] = run;
            run += v;
        }
    if (t == P3_THREADS - 1) out[n] = run;
    __syncthreads();
}

// ---------------------------------------------------------------------------
// push + deposit
// ---------------------------------------------------------------------------
// A pencil's markers are walked in chunks of at most NB markers, each inside
// one segment; the marker fields of the next chunk are staged into shared
// memory by bulk copies (TMA) while the current one is processed.
template <typename T>
struct Stage3 {
    static constexpr int NB = P3_THREADS * Cfg3<T>::MPT;   // markers per chunk
    // staged fields: FP32 cell, offset, v_x, v_y, v_z, f; FP64 x, v_x, f (the
    // weights of the (v_y, v_z) cells are stored beside the marker)
    static constexpr int NF = sizeof(T) == 4 ? 6 : 3;
    static constexpr int FVX = sizeof(T) == 4 ? 2 : 1;       // staged field of v_x
    static constexpr int FF = NF - 1;                         // staged field of f
    // the balanced gather (column accumulators in shared-memory row planes,
    // columns sorted by their pair counts): the FP64 form, whose instructions
    // cost an SM sub-partition the same whatever their active lanes
    static constexpr bool BAL = sizeof(T) == 8;
    static constexpr int AL = 16 / (int)sizeof(T);           // markers per 16 bytes
    static constexpr int SLEN = NB + 2 * AL;                 // staged entries per field
};

// FP64 gather (see k_pd3): count buckets of the columns' pair counts; the
// gather's column blocks are laid out for eight warps
constexpr int GBK = 64;
// FP64: the short remainder (fewer markers) of a segment just over NB
// markers skips the x sort and the gather: its markers deposit by global
// reductions like the markers off their row, which saves the phases of the
// sort (scan, scatter, column order) and their barriers for a handful of
// markers (in FP32 the gather of a few markers costs less than their global
// reductions)
constexpr int P3_TAIL = 96;
constexpr int GL = 128;   // gather lanes: one warp per SM sub-partition
static_assert(P3_THREADS >= GL && GL % 32 == 0, "k_pd3's FP64 gather needs GL threads");

// FP64: the two row planes of the column accumulators, the column order and
// the count buckets, after the integer arrays (16-byte aligned)
template <typename T>
static size_t pd3_acc_offset(int nx, int nkey)
{
    using S = Stage3<T>;
    size_t b = 2 * (size_t)S::NF * S::SLEN * sizeof(T);      // two staging buffers
    b += sizeof(T) * (7 * (size_t)S::NB + nx);                 // sorted payload, E
    b += 4 * (2 * (size_t)nx + 1) + 4 * ((size_t)nkey + 2) + 64;   // histogram, bin starts, segment row
    return (b + 15) / 16 * 16;
}

template <typename T>
static size_t pd3_bytes(int nx, int nkey)
{
    size_t b = pd3_acc_offset<T>(nx, nkey);
    if (Stage3<T>::BAL) b += 2 * 8 * (size_t)nx * sizeof(T) + 4 * (size_t)nx + 8 * (size_t)GBK + 16;
    return (b + 15) / 16 * 16;
}

size_t pd3_smem_bytes(int nx, int nkey, int prec)
{
    return prec == AVL_FP32 ? pd3_bytes<float>(nx, nkey) : pd3_bytes<double>(nx, nkey);
}

// largest key count (nv[0] + 1) over the species of a context
static int nkey_max(const StepArgs& h)
{
    int m = 2;
    for (int s = 0; s < h.ns; ++s) m = std::max(m, h.sp[s].nv[0] + 1);
    return m;
}

// weights of the pencil's four (v_y, v_z) cells: (jy, jz), (jy+1, jz),
// (jy, jz+1), (jy+1, jz+1)
template <typename T>
__device__ __forceinline__ void plane_weights(T wy, T wz, T (&q)[4])
{
    const T ya = (T)1 - wy, za = (T)1 - wz;
    q[0] = ya * za;
    q[1] = wy * za;
    q[2] = ya * wz;
    q[3] = wy * wz;
}

// FP64: the weights of a marker's four (v_y, v_z) cells, stored beside the
// marker (they change only when a magnetic field turns v): the plane weights
// of its dual cells, or 0 when its footprint misses the grid in v_y or v_z
// (such a marker sits in a clamped pencil and deposits nothing)
template <typename T>
__device__ __forceinline__ void marker_planes(const VCoef<T>& vc, T vy, T vz, T (&wq)[4])
{
    T wy, wz;
    const int jy = dual3(vy, vc.a[1], vc.b[1], vc.n[1], wy);
    const int jz = dual3(vz, vc.a[2], vc.b[2], vc.n[2], wz);
    if (jy < -1 || jy >= vc.n[1] || jz < -1 || jz >= vc.n[2]) {
        wq[0] = wq[1] = wq[2] = wq[3] = (T)0;
        return;
    }
    plane_weights(wy, wz, wq);
}

__device__ __forceinline__ void store_planes(void* mwq, long long k, const double (&wq)[4])
{
    double2* p = reinterpret_cast<double2*>(mwq) + 2 * k;
    p[0] = make_double2(wq[0], wq[1]);
    p[1] = make_double2(wq[2], wq[3]);
}

// the pencil's four (v_y, v_z) planes: first grid offset of each (row 0,
// column 0) and whether it lies on the grid
struct Planes {
    int base[4];
    bool ok[4];
};

// A marker whose v_x dual row j is not its segment's deposits its 16
// cloud-in-cell contributions apart from the gather, straight into the
// global accumulator.  This is one of them: corner bits x (bit 0), v_x row
// (bit 1), (v_y, v_z) plane (bits 2-3).
template <typename T>
__device__ __forceinline__ void deposit_corner_q(T* gacc, int cells, const Planes& pl, int nx, int nvx, int bin, T u,
                                                 int j, T w, T wqv, T f, int corner)
{
    const int cx = corner & 1, cv = (corner >> 1) & 1, q = corner >> 2;
    const bool okq = q == 0 ? pl.ok[0] : q == 1 ? pl.ok[1] : q == 2 ? pl.ok[2] : pl.ok[3];
    const int row = j + cv;
    if (!okq || row < 0 || row >= nvx) return;
    const int x = cx ? (bin + 1 == nx ? 0 : bin + 1) : bin;
    const T ax = cx ? u : (T)1 - u;
    const T a = ax * (cv ? w : (T)1 - w) * wqv;
    if (a == (T)0) return;
    const int base = q == 0 ? pl.base[0] : q == 1 ? pl.base[1] : q == 2 ? pl.base[2] : pl.base[3];
    const int o = base + row * nx + x;
    atomicAdd(gacc + o, a * f);
    atomicAdd(gacc + cells + o, a);
}

// FP32: the plane weight from the marker's (v_y, v_z) cell weights
template <typename T>
__device__ __forceinline__ void deposit_corner(T* gacc, int cells, const Planes& pl, int nx, int nvx, int bin, T u,
                                               int j, T w, T wy, T wz, T f, int corner)
{
    const int q = corner >> 2;
    const T ay = (q & 1) ? wy : (T)1 - wy, az = (q & 2) ? wz : (T)1 - wz;
    deposit_corner_q<T>(gacc, cells, pl, nx, nvx, bin, u, j, w, ay * az, f, corner);
}

// exclusive scan of hist[0, nx) into start[0, nx], start[nx] = total; each
// thread owns CPT consecutive bins and clears them for the next chunk
template <int CPT>
__device__ __forceinline__ void chunk_scan(int* hist, int* start, int nx, int* wsum)
{
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int i0 = t * CPT;
    int v[CPT], loc = 0;
#pragma unroll
    for (int i = 0; i < CPT; ++i) {
        v[i] = i0 + i < nx ? hist[i0 + i] : 0;
        loc += v[i];
    }
    int incl = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    int pre = 0;
    for (int w = 0; w < warp; ++w) pre += wsum[w];
    int run = pre + incl - loc;
#pragma unroll
    for (int i = 0; i < CPT; ++i) {
        if (i0 + i < nx) {
            start[i0 + i] = run;
            hist[i0 + i] = 0;
        }
        run += v[i];
    }
    if (i0 < nx && nx <= i0 + CPT) start[nx] = run;
    __syncthreads();
}

// mode 0: deposit of the current markers of every species (refresh);
// mode 1: push of the mobile species, then deposit of the new state;
// mode 2: deposit of the mobile species (pushed and re-sorted before).
// PUSH (mode 1) is a template parameter so that the deposit-only instances
// keep their own register budget (FP32, one column per thread: three CTAs
// per SM with the push, four without).
template <typename T, int CPT, bool PUSH>
__global__ void __launch_bounds__(P3_THREADS, sizeof(T) == 4 ? (CPT == 1 ? (PUSH ? 3 : 4) : (CPT == 2 ? 2 : 1))
                                                             : (CPT == 1 ? 2 : 1))
    k_pd3(const StepArgs* __restrict__ A, int mode)
{
    using S = Stage3<T>;
    constexpr int MPT = Cfg3<T>::MPT;
    constexpr int NB = S::NB, NF = S::NF, AL = S::AL, SLEN = S::SLEN;
    constexpr int FVX = S::FVX, FF = S::FF;   // staged fields of v_x and f (FP32: v_y, v_z between)
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint64_t bar[2];
    __shared__ int wsum[P3_THREADS / 32];
    __shared__ unsigned long long mov_s, far_s;
    __shared__ int flag_s;
    __shared__ int nmv_s;
    __shared__ const void* src_s[6];

    const int g = blockIdx.x;
    const int s = species_of_pen(A, g);
    const SpDev& sp = A->sp[s];
    constexpr bool push = PUSH;   // mode == 1
    if (mode != 0 && !sp.mobile) return;
    Ctl* ctl = A->ctl;
    const long long wait_first = ctl->wait_limit;
    const int p = g - sp.pen_base;
    const int nx = sp.nx, nvx = sp.nv[0], nvy = sp.nv[1], nvz = sp.nv[2], nkey = sp.nkey;
    const int pjy = p % (nvy + 1) - 1, pjz = p / (nvy + 1) - 1;
    const int cb = ctl->cur[s];
    const int cells = sp.nvflat * nx;
    T* const gacc = reinterpret_cast<T*>(sp.acc[ctl->asel[s]]);
    const int* segg = sp.seg[cb] + (size_t)p * (nkey + 1);

    // shared memory: staging | payload (7 x NB) | E | hist | start | segment row
    T* stage = reinterpret_cast<T*>(smem);
    T* pay = stage + 2 * NF * SLEN;
    T* Es = pay + 7 * NB;
    int* hist = reinterpret_cast<int*>(Es + nx);
    int* start = hist + nx;
    int* segs = start + nx + 1;
    // balanced gather (FP64): column accumulators of rows jseg, jseg + 1 in
    // two planes of 8 x nx (entry e of column x: plane[e * nx + x]), the
    // columns in order of their pair counts, the count buckets and their
    // first positions
    const size_t acc_off = (((size_t)(reinterpret_cast<unsigned char*>(segs + nkey + 2) - smem)) + 15) / 16 * 16;
    T* RA = reinterpret_cast<T*>(smem + acc_off);
    int* ordc = reinterpret_cast<int*>(RA + 2 * 8 * nx);
    int* gbk = ordc + nx;
    int* gbase = gbk + GBK;

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        mov_s = 0;
        far_s = 0;
        flag_s = 0;
        nmv_s = 0;
        if constexpr (sizeof(T) == 4) {
            src_s[0] = sp.mx[cb];
            src_s[1] = sp.moff[cb];
        } else {
            src_s[0] = sp.mx[cb];
        }
        src_s[FVX] = sp.mv[cb][0];
        if constexpr (sizeof(T) == 4) {
            src_s[FVX + 1] = sp.mv[cb][1];
            src_s[FVX + 2] = sp.mv[cb][2];
        }
        src_s[FF] = sp.mf[cb];
    }
    for (int i = threadIdx.x; i < nx; i += P3_THREADS) {
        hist[i] = 0;
        if (push) Es[i] = sizeof(T) == 4 ? (T)A->fd.E32[i] : (T)A->fd.E64[i];
    }
    for (int i = threadIdx.x; i <= nkey; i += P3_THREADS) segs[i] = segg[i];
    if constexpr (S::BAL) {
        for (int i = threadIdx.x; i < 2 * 8 * nx; i += P3_THREADS) RA[i] = 0.0;
        for (int i = threadIdx.x; i < GBK; i += P3_THREADS) gbk[i] = 0;
    }
    __syncthreads();

    // bulk copy of the chunk [b, b + cnt) of every staged field into buffer bf
    auto issue = [&](int bf, int b, int cnt) {
        const int a0 = b & ~(AL - 1);
        const int a1 = (b + cnt + AL - 1) & ~(AL - 1);
        const unsigned bytes = (unsigned)(a1 - a0) * (unsigned)sizeof(T);
        mbar_arrive_expect_tx(&bar[bf], bytes * NF);
        for (int f = 0; f < NF; ++f)
            bulk_g2s(stage + (bf * NF + f) * SLEN, reinterpret_cast<const T*>(src_s[f]) + a0, bytes, &bar[bf]);
    };
    // first chunk at or after key k whose segment is not empty
    auto first_from = [&](int k, int& kb) {
        for (; k < nkey; ++k)
            if (segs[k] < segs[k + 1]) break;
        kb = k < nkey ? segs[k] : 0;
        return k;
    };
    if (threadIdx.x == 0) {
        int b;
        const int k0 = first_from(0, b);
        if (k0 < nkey) issue(0, b, min(NB, segs[k0 + 1] - b));
    }

    // cached marker pointers (in-place write back)
    T* const gvx = reinterpret_cast<T*>(sp.mv[cb][0]);
    void* const gx = sp.mx[cb];
    float* const goff = sp.moff[cb];
    VCoef<T> vc;
    vc.init(sp);
    const T qm_dt = (T)sp.qm_dt, dt_dx = (T)sp.dt_dx;
    const double dt_dx52 = sp.dt_dx * PosX::ONE;   // FP64: dt / dx in 2^-52 cells
    Planes pl;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int ky = pjy + (q & 1), kz = pjz + (q >> 1);
        pl.ok[q] = ky >= 0 && ky < nvy && kz >= 0 && kz < nvz;
        pl.base[q] = pl.ok[q] ? (kz * nvy + ky) * nvx * nx : 0;
    }

    // register rows: Rm = row jseg - 1, R0 = row jseg, R1 = row jseg + 1;
    // entry 2q: numerator, 2q + 1: denominator of plane q
    T Rm[CPT][8], R0[CPT][8], R1[CPT][8];
#pragma unroll
    for (int c = 0; c < CPT; ++c)
#pragma unroll
        for (int e = 0; e < 8; ++e) Rm[c][e] = R0[c][e] = R1[c][e] = (T)0;
    unsigned long long nmov = 0, nfar = 0;
    int buf = 0;
    unsigned ph0 = 0, ph1 = 0;
    int rp = 0;   // FP64: plane of row jseg (the other holds row jseg + 1)

    for (int k = 0; k < nkey; ++k) {
        const int jseg = k - 1;
        const int send = segs[k + 1];
        for (int b0 = segs[k]; b0 < send; b0 += NB) {
            const int cnt = min(NB, send - b0);
            const bool tail = S::BAL && b0 > segs[k] && cnt < P3_TAIL;   // FP64: the remainder of a segment over NB
            // stage the next chunk into the other buffer (free since the end of
            // the previous chunk)
            if (threadIdx.x == 0) {
                int nk = k, nb = b0 + NB;
                if (nb >= send) nk = first_from(k + 1, nb);
                if (nk < nkey) issue(buf ^ 1, nb, min(NB, segs[nk + 1] - nb));
            }
            // FP64: the stored (v_y, v_z) cell weights of this chunk's markers,
            // loaded while its staged fields are in flight
            double2 qlo[MPT], qhi[MPT];
            if constexpr (sizeof(T) == 8) {
                const double2* wqg = reinterpret_cast<const double2*>(sp.mwq[cb]);
#pragma unroll
                for (int m = 0; m < MPT; ++m) {
                    const int i = m * P3_THREADS + threadIdx.x;
                    qlo[m] = qhi[m] = make_double2(0.0, 0.0);
                    if (i < cnt) {
                        qlo[m] = wqg[2 * (long long)(b0 + i)];
                        qhi[m] = wqg[2 * (long long)(b0 + i) + 1];
                    }
                }
            }
            const unsigned ph = buf ? ph1 : ph0;
            if (!mbar_wait_or_drain(&bar[buf], ph, wait_first, WAIT_LIMIT)) flag_s = 1;
            if (buf) ph1 ^= 1u; else ph0 ^= 1u;
            const T* st = stage + buf * NF * SLEN;
            const int o0 = b0 & (AL - 1);

            T pu[MPT], pw[MPT], pf[MPT], py[MPT], pz[MPT];
            int pbin[MPT], prank[MPT];
#pragma unroll
            for (int m = 0; m < MPT; ++m) {
                prank[m] = -1;
                pbin[m] = 0;
                const int i = m * P3_THREADS + threadIdx.x;
                if (i >= cnt) continue;
                const int si = o0 + i;
                const int idx = b0 + i;
                Pos3<T> pos;
                if constexpr (sizeof(T) == 4) {
                    pos.c = reinterpret_cast<const int*>(st)[si];
                    pos.o = st[SLEN + si];
                } else {
                    pos.X = reinterpret_cast<const long long*>(st)[si];
                }
                T vx = st[FVX * SLEN + si];
                if (push) {
                    int i0;
                    T wx;
                    pos.cic(i0, wx);
                    int ia, ib;
                    wrap_pair(i0, nx, ia, ib);
                    if constexpr (sizeof(T) == 8) {
                        // FP64 (the FP64 pipe limits this form): E_a + w (E_b - E_a)
                        // fused, one FP64 operation fewer than the plain form;
                        // the displacement in 2^-52 cells (dt_dx52 = dt / dx 2^52)
                        const T Ea = Es[ia];
                        vx = fma(qm_dt, fma(wx, Es[ib] - Ea, Ea), vx);
                        pos.drift_scaled(vx * dt_dx52, nx);
                    } else {
                        const T El = ((T)1 - wx) * Es[ia] + wx * Es[ib];
                        vx = vx + qm_dt * El;
                        pos.drift(vx * dt_dx, nx);
                    }
                    if constexpr (sizeof(T) == 4) {
                        reinterpret_cast<int*>(gx)[idx] = pos.c;
                        goff[idx] = pos.o;
                    } else {
                        reinterpret_cast<long long*>(gx)[idx] = pos.X;
                    }
                    gvx[idx] = vx;
                }
                const T f = st[FF * SLEN + si];
                T wy = (T)0, wz = (T)0, w;
                // FP32: the (v_y, v_z) dual cells, checked against the pencil;
                // FP64: the stored cell weights (0 for a footprint off the grid)
                if constexpr (sizeof(T) == 4) {
                    const int jy = dual3(st[(FVX + 1) * SLEN + si], vc.a[1], vc.b[1], vc.n[1], wy);
                    const int jz = dual3(st[(FVX + 2) * SLEN + si], vc.a[2], vc.b[2], vc.n[2], wz);
                    if (jy != pjy || jz != pjz) {
                        // outside the pencil only when the footprint misses the grid
                        if (jy >= -1 && jy < nvy && jz >= -1 && jz < nvz) flag_s |= 2;
                        continue;
                    }
                }
                const int jx = dual3(vx, vc.a[0], vc.b[0], nvx, w);
                if (jx < -1 || jx >= nvx) continue;
                int i0;
                T u;
                pos.cic(i0, u);
                int bin = i0 < 0 ? i0 + nx : i0;
                bin = min(max(bin, 0), nx - 1);
                const int d = jx - jseg;
                if (d == 0 && !tail) {
                    prank[m] = atomicAdd(&hist[bin], 1);
                } else {
                    // off its segment's row (or in a short chunk): parked at the
                    // tail of the payload arrays (the stays fill them from the
                    // front) and deposited by the whole block after the sort
                    if (d != 0) {
                        ++nmov;
                        if (d > 1 || d < -1) ++nfar;
                    }
                    const int o = NB - 1 - atomicAdd(&nmv_s, 1);
                    pay[0 * NB + o] = u;
                    pay[1 * NB + o] = w;
                    pay[2 * NB + o] = f;
                    if constexpr (sizeof(T) == 4) {
                        pay[3 * NB + o] = wy;
                        pay[4 * NB + o] = wz;
                    } else {
                        pay[3 * NB + o] = (T)idx;   // FP64: its stored cell weights are read by index
                    }
                    pay[5 * NB + o] = (T)bin;
                    pay[6 * NB + o] = (T)jx;
                }
                pbin[m] = bin;
                pu[m] = u;
                pw[m] = w;
                pf[m] = f;
                py[m] = wy;
                pz[m] = wz;
            }
            __syncthreads();
            const int nmv = nmv_s;
            // the parked markers: one thread per (marker, corner) into the global
            // accumulator, so that a chunk's few movers do not hold one warp
            // behind the others at the chunk's barrier
            auto deposit_parked = [&]() {
                for (int t = threadIdx.x; t < nmv * 16; t += P3_THREADS) {
                    const int o = NB - 1 - (t >> 4);
                    const int jx = (int)pay[6 * NB + o];
                    if constexpr (sizeof(T) == 4) {
                        deposit_corner<T>(gacc, cells, pl, nx, nvx, (int)pay[5 * NB + o], pay[0 * NB + o], jx,
                                          pay[1 * NB + o], pay[3 * NB + o], pay[4 * NB + o], pay[2 * NB + o],
                                          t & 15);
                    } else {
                        const long long mi = (long long)pay[3 * NB + o];
                        const T wqv = reinterpret_cast<const double*>(sp.mwq[cb])[4 * mi + ((t & 15) >> 2)];
                        deposit_corner_q<T>(gacc, cells, pl, nx, nvx, (int)pay[5 * NB + o], pay[0 * NB + o], jx,
                                            pay[1 * NB + o], wqv, pay[2 * NB + o], t & 15);
                    }
                }
            };
            if (tail) {
                __syncthreads();   // every thread has read nmv_s
                if (threadIdx.x == 0) nmv_s = 0;
                deposit_parked();
                __syncthreads();
                buf ^= 1;
                continue;
            }
            chunk_scan<CPT>(hist, start, nx, wsum);   // every thread has read nmv_s by its barriers
            if (threadIdx.x == 0) nmv_s = 0;
            // stays into x-sorted order
#pragma unroll
            for (int m = 0; m < MPT; ++m) {
                if (prank[m] < 0) continue;
                const int o = start[pbin[m]] + prank[m];
                T wq[4];
                if constexpr (sizeof(T) == 4) {
                    plane_weights(py[m], pz[m], wq);
                } else {
                    wq[0] = qlo[m].x;
                    wq[1] = qlo[m].y;
                    wq[2] = qhi[m].x;
                    wq[3] = qhi[m].y;
                }
                pay[0 * NB + o] = pu[m];
                pay[1 * NB + o] = pw[m];
                pay[2 * NB + o] = pf[m];
#pragma unroll
                for (int q = 0; q < 4; ++q) pay[(3 + q) * NB + o] = wq[q];
            }
            // FP64: pairs (marker, column) of each column = the markers of its
            // two dual cells; the columns are counting-sorted by that count
            // so that a warp's lanes loop over nearly equal counts (an FP64
            // warp instruction costs its sub-partition the same whatever the
            // number of active lanes)
            int gb[CPT], grank[CPT];
            if constexpr (S::BAL) {
#pragma unroll
                for (int c = 0; c < CPT; ++c) {
                    const int x = threadIdx.x + c * P3_THREADS;
                    gb[c] = -1;
                    if (x >= nx) continue;
                    const int xm = x == 0 ? nx - 1 : x - 1;
                    const int cnt = (start[xm + 1] - start[xm]) + (start[x + 1] - start[x]);
                    gb[c] = min(cnt, GBK - 1);
                    grank[c] = atomicAdd(&gbk[gb[c]], 1);
                }
            }
            __syncthreads();
            if constexpr (S::BAL) {
                if (threadIdx.x < 32) {   // exclusive scan of the buckets (two per lane)
                    const int lane = threadIdx.x;
                    const int a0 = gbk[2 * lane], a1 = gbk[2 * lane + 1];
                    int incl = a0 + a1;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += y;
                    }
                    gbase[2 * lane] = incl - a0 - a1;
                    gbase[2 * lane + 1] = incl - a1;
                }
            }
            deposit_parked();
            // gather: column x takes weight u from the markers of dual cell
            // x - 1 and 1 - u from those of dual cell x, which follow them in
            // the sorted order (one loop; two at the periodic seam)
            if constexpr (S::BAL) {
                __syncthreads();
#pragma unroll
                for (int c = 0; c < CPT; ++c)
                    if (gb[c] >= 0) ordc[gbase[gb[c]] + grank[c]] = threadIdx.x + c * P3_THREADS;
                __syncthreads();
                for (int i = threadIdx.x; i < GBK; i += P3_THREADS) gbk[i] = 0;
                T* P0 = RA + (size_t)rp * 8 * nx;
                T* P1 = RA + (size_t)(rp ^ 1) * 8 * nx;
                // gather lanes: the first GL threads (one warp per SM
                // sub-partition) each take the sorted columns l and 2K - 1 - l
                // (then 2K + l, 4K - 1 - l, ...), a light and a heavy one, and
                // walk their pairs in one loop, so that the lanes of a warp do
                // nearly equal work; a lane's accumulators go back to the row
                // planes when its column changes.  Each column is summed in
                // pair order (dual cell x - 1, then dual cell x).
                const int K = min(GL, (nx + 1) >> 1);
                const int l = threadIdx.x;
                if (l < K) {
                    int r = 0, x = -1, lo = 0, nup = 0, blo = 0, n = 0, kr = 0;
                    T A0[8], A1[8];
                    for (;;) {
                        if (kr == n) {
                            if (x >= 0) {
#pragma unroll
                                for (int e = 0; e < 8; ++e) {
                                    P0[e * nx + x] = A0[e];
                                    P1[e * nx + x] = A1[e];
                                }
                            }
                            x = -1;
                            while (r * K < nx) {
                                const int pos = r * K + ((r & 1) ? K - 1 - l : l);
                                ++r;
                                if (pos >= nx) continue;
                                const int cx = ordc[pos];
                                const int cxm = cx == 0 ? nx - 1 : cx - 1;
                                const int a0 = start[cxm], a1 = start[cxm + 1];
                                const int b0 = start[cx], b1 = start[cx + 1];
                                if (a1 - a0 + b1 - b0 == 0) continue;
                                x = cx;
                                lo = a0;
                                nup = a1 - a0;
                                blo = b0;
                                n = nup + b1 - b0;
                                kr = 0;
                                break;
                            }
                            if (x < 0) break;
#pragma unroll
                            for (int e = 0; e < 8; ++e) {
                                A0[e] = P0[e * nx + x];
                                A1[e] = P1[e * nx + x];
                            }
                        }
                        const bool upper = kr < nup;
                        const int i = upper ? lo + kr : blo + (kr - nup);
                        ++kr;
                        const T u = pay[i];
                        const T ax = upper ? u : (T)1 - u;
                        const T a1 = ax * pay[NB + i];
                        const T a0 = ax - a1;
                        const T f = pay[2 * NB + i];
                        const T f0 = a0 * f, f1 = a1 * f;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const T wqv = pay[(3 + q) * NB + i];
                            A0[2 * q] += f0 * wqv;
                            A0[2 * q + 1] += a0 * wqv;
                            A1[2 * q] += f1 * wqv;
                            A1[2 * q + 1] += a1 * wqv;
                        }
                    }
                }
            } else
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int x = threadIdx.x + c * P3_THREADS;
                if (x >= nx) continue;
                const int xm = x == 0 ? nx - 1 : x - 1;
                const int mid = start[x];
                const int lo0 = start[xm], hi0 = x == 0 ? start[nx] : mid;
                const int hi1 = start[x + 1];
                for (int pass = 0; pass < (x == 0 ? 2 : 1); ++pass) {
                    const int lo = pass ? mid : lo0, hi = (x == 0 && !pass) ? hi0 : hi1;
                    for (int i = lo; i < hi; ++i) {
                        const T u = pay[i];
                        const bool upper = x == 0 ? pass == 0 : i < mid;
                        const T ax = upper ? u : (T)1 - u;
                        const T a1 = ax * pay[NB + i];
                        const T a0 = ax - a1;
                        const T f = pay[2 * NB + i];
                        const T f0 = a0 * f, f1 = a1 * f;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const T wqv = pay[(3 + q) * NB + i];
                            R0[c][2 * q] += f0 * wqv;
                            R0[c][2 * q + 1] += a0 * wqv;
                            R1[c][2 * q] += f1 * wqv;
                            R1[c][2 * q + 1] += a1 * wqv;
                        }
                    }
                }
            }
            __syncthreads();
            buf ^= 1;
        }
        if constexpr (S::BAL) {
            // row jseg is complete (the next segment reaches rows jseg + 1 and
            // jseg + 2): its plane into the global accumulator and cleared,
            // then the planes swap
            T* P0 = RA + (size_t)rp * 8 * nx;
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int x = threadIdx.x + c * P3_THREADS;
                if (x >= nx) continue;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const T vn = P0[(2 * q) * nx + x], vd = P0[(2 * q + 1) * nx + x];
                    if (jseg >= 0 && jseg < nvx && pl.ok[q] && __double_as_longlong(vd) != 0) {
                        const int o = pl.base[q] + jseg * nx + x;
                        atomicAdd(gacc + o, vn);
                        atomicAdd(gacc + cells + o, vd);
                    }
                    P0[(2 * q) * nx + x] = (T)0;
                    P0[(2 * q + 1) * nx + x] = (T)0;
                }
            }
            rp ^= 1;
            __syncthreads();
            continue;
        }
        // row jseg - 1 is complete (no later segment reaches it): registers into
        // the global accumulator; then rotate the rows
        const int row = jseg - 1;
        if (row >= 0) {
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int x = threadIdx.x + c * P3_THREADS;
                if (x >= nx) continue;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const T vn = Rm[c][2 * q], vd = Rm[c][2 * q + 1];
                    if (pl.ok[q] && vd != (T)0) {
                        const int o = pl.base[q] + row * nx + x;
                        atomicAdd(gacc + o, vn);
                        atomicAdd(gacc + cells + o, vd);
                    }
                }
            }
        }
#pragma unroll
        for (int c = 0; c < CPT; ++c)
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                Rm[c][e] = R0[c][e];
                R0[c][e] = R1[c][e];
                R1[c][e] = (T)0;
            }
        __syncthreads();
    }
    // the last row (nvx - 1) after the last segment
    if constexpr (!S::BAL) {
        const int row = nvx - 1;
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const int x = threadIdx.x + c * P3_THREADS;
            if (x >= nx) continue;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const T vn = Rm[c][2 * q];
                const T vd = Rm[c][2 * q + 1];
                if (pl.ok[q] && vd != (T)0) {
                    const int o = pl.base[q] + row * nx + x;
                    atomicAdd(gacc + o, vn);
                    atomicAdd(gacc + cells + o, vd);
                }
            }
        }
    }

    if (nmov) atomicAdd(&mov_s, nmov);
    if (nfar) atomicAdd(&far_s, nfar);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (mov_s) atomicAdd(&ctl->movers[s], mov_s);
        if (far_s) atomicAdd(&ctl->far_movers[s], far_s);
        if (flag_s & 2) atomicOr(&ctl->err, ERR_CAPACITY);
        if (flag_s & 1) atomicOr(&ctl->err, ERR_TIMEOUT);
    }
}

// ---------------------------------------------------------------------------
// finalize: f = num / den (Eq. 4), charge per row group (Eq. 14), diagnostics
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(FIN3_X * FIN3_R) k_fin3(const StepArgs* __restrict__ A, int all_species)
{
    constexpr int NT = FIN3_X * FIN3_R;
    __shared__ double col_red[FIN3_R][FIN3_X];
    __shared__ double red[3][NT / 32];
    const int g = blockIdx.x;
    const int s = species_of_fin3(A, g);
    const SpDev& sp = A->sp[s];
    if (!all_species && !sp.mobile) return;
    const int blk = g - sp.fin_base;
    const int xb = blk % sp.nxb, rqi = blk / sp.nxb;
    const int nx = sp.nx, nvf = sp.nvflat;
    const int col = threadIdx.x % FIN3_X, lr = threadIdx.x / FIN3_X;
    const int x = xb * FIN3_X + col;
    const bool xok = x < nx;
    const int j0 = rqi * sp.rq, j1 = min(nvf, j0 + sp.rq);
    const int a = A->ctl->asel[s];
    const size_t cells = (size_t)nvf * nx;
    const T* num = reinterpret_cast<const T*>(sp.acc[a]);
    const T* den = num + cells;
    T* clr = reinterpret_cast<T*>(sp.acc[1 - a]);
    T* fg = reinterpret_cast<T*>(sp.fgrid);
    const T* v2 = reinterpret_cast<const T*>(sp.v2row);
    ColAcc<T> acc;
    if constexpr (sizeof(T) == 8) acc.logtab = A->fd.logtab;
    auto cell = [&](int j, T nn, T dd, T v2j) {
        const size_t o = (size_t)j * nx + x;
        T f;
        if constexpr (sizeof(T) == 8)
            f = __double_as_longlong(dd) > 0 ? div_nr(nn, dd) : 0.0;   // dd >= 0 is a sum of weights
        else
            f = dd > (T)0 ? nn / dd : (T)0;
        fg[o] = f;
        clr[o] = (T)0;
        clr[cells + o] = (T)0;
        acc.add(f, (T)0, v2j);
    };
    if (xok) {
        // four rows per iteration, their loads issued together; the cells
        // are still taken in row order
        int j = j0 + lr;
        for (; j + 3 * FIN3_R < j1; j += 4 * FIN3_R) {
            T nn[4], dd[4], vv[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const size_t o = (size_t)(j + k * FIN3_R) * nx + x;
                nn[k] = num[o];
                dd[k] = den[o];
                vv[k] = v2[j + k * FIN3_R];
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) cell(j + k * FIN3_R, nn[k], dd[k], vv[k]);
        }
        for (; j < j1; j += FIN3_R) {
            const size_t o = (size_t)j * nx + x;
            cell(j, num[o], den[o], v2[j]);
        }
    }
    const double dvol = sp.dv[0] * sp.dv[1] * sp.dv[2];
    col_red[lr][col] = acc.r();
    __syncthreads();
    if (lr == 0 && xok) {
        double r = 0.0;
        for (int k = 0; k < FIN3_R; ++k) r += col_red[k][col];
        sp.rho_part[(size_t)rqi * nx + x] = sp.q * dvol * r;
    }
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
        double n0 = 0, w0 = 0, s0 = 0;
        for (int w = 0; w < NT / 32; ++w) {
            n0 += red[0][w];
            w0 += red[1][w];
            s0 += red[2][w];
        }
        const double cell = sp.dx * dvol;
        sp.dpart[(size_t)blk * 4 + 0] = n0 * cell;
        sp.dpart[(size_t)blk * 4 + 1] = 0.5 * sp.m * w0 * cell;
        sp.dpart[(size_t)blk * 4 + 2] = s0 * cell;
        sp.dpart[(size_t)blk * 4 + 3] = 0.0;
    }
}

// ---------------------------------------------------------------------------
// re-sort: every pencil of a species the field kernel marked, from buffer
// 1 - cur into buffer cur (the field kernel has already flipped cur)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(P3_THREADS) k_sort3(const StepArgs* __restrict__ A)
{
    __shared__ int cnt[NV3_MAX + 2];
    __shared__ int wsum[P3_THREADS / 32];
    const int g = blockIdx.x;
    const int s = species_of_pen(A, g);
    const SpDev& sp = A->sp[s];
    const Ctl* ctl = A->ctl;
    if (!sp.mobile || !ctl->sort_now[s]) return;
    const int p = g - sp.pen_base;
    const int dst = ctl->cur[s], src = 1 - dst;
    const int nk = sp.nkey, nvx = sp.nv[0];
    const int* sg = sp.seg[src] + (size_t)p * (nk + 1);
    int* dg = sp.seg[dst] + (size_t)p * (nk + 1);
    const int beg = sg[0], end = sg[nk];
    T ax, bx;
    dual_coef<T>(sp, 0, ax, bx);
    const T* vxs = reinterpret_cast<const T*>(sp.mv[src][0]);
    for (int i = threadIdx.x; i < nk + 1; i += P3_THREADS) cnt[i] = 0;
    __syncthreads();
    for (int b0 = beg; b0 < end; b0 += P3_THREADS) {
        const int k = b0 + threadIdx.x;
        const bool ok = k < end;
        int key = 0;
        if (ok) {
            T w;
            key = key_of(dual3(vxs[k], ax, bx, nvx, w), nvx);
        }
        const int kk = ok ? key : -1;
        const unsigned grp = __match_any_sync(0xffffffffu, kk);
        if (ok && (threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(&cnt[key], __popc(grp));
    }
    __syncthreads();
    block_exscan(cnt, cnt, nk, (nk + P3_THREADS - 1) / P3_THREADS, wsum);
    for (int i = threadIdx.x; i <= nk; i += P3_THREADS) dg[i] = beg + cnt[i];
    __syncthreads();
    for (int b0 = beg; b0 < end; b0 += P3_THREADS) {
        const int k = b0 + threadIdx.x;
        const bool ok = k < end;
        int key = 0;
        T vx = 0;
        if (ok) {
            T w;
            vx = vxs[k];
            key = key_of(dual3(vx, ax, bx, nvx, w), nvx);
        }
        const int slot = beg + warp_slot(cnt, key, ok);
        if (ok && slot >= beg && slot < end) {
            Pos3<T> pos;
            pos.load(sp, src, k);
            pos.store(sp, dst, slot);
            reinterpret_cast<T*>(sp.mv[dst][0])[slot] = vx;
            reinterpret_cast<T*>(sp.mv[dst][1])[slot] = reinterpret_cast<const T*>(sp.mv[src][1])[k];
            reinterpret_cast<T*>(sp.mv[dst][2])[slot] = reinterpret_cast<const T*>(sp.mv[src][2])[k];
            reinterpret_cast<T*>(sp.mf[dst])[slot] = reinterpret_cast<const T*>(sp.mf[src])[k];
            if constexpr (sizeof(T) == 8) {
                const double2* ps = reinterpret_cast<const double2*>(sp.mwq[src]) + 2 * (long long)k;
                double2* pd = reinterpret_cast<double2*>(sp.mwq[dst]) + 2 * (long long)slot;
                pd[0] = ps[0];
                pd[1] = ps[1];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// marker creation: jittered lattice (Sec. 2 / Sec. 3.1) or caller arrays,
// counting-sorted by (pencil, key) into buffer 0
// ---------------------------------------------------------------------------
struct MarkerIn3 {
    double xi;   // position in cells
    double v[3];
    double f;
    bool ok;
};

// lattice marker number k in generation order (v_z, v_y, v_x cell slowest,
// then x cell, then sub-point); the jitter streams use the row-major marker
// number ((((i nvx + jx) nvy + jy) nvz + jz) ppc + sub)
struct LatticeSrc3 {
    const avl_f0* f0;
    unsigned long long seed;
    double jitter;
    int s;
    int l[4];
    __device__ MarkerIn3 get(const SpDev& sp, long long k) const
    {
        const int ppc = l[0] * l[1] * l[2] * l[3];
        const int sub = (int)(k % ppc);
        long long r = k / ppc;
        const int i = (int)(r % sp.nx);
        r /= sp.nx;
        const int jx = (int)(r % sp.nv[0]);
        r /= sp.nv[0];
        const int jy = (int)(r % sp.nv[1]);
        const int jz = (int)(r / sp.nv[1]);
        const long long cell = (((long long)i * sp.nv[0] + jx) * sp.nv[1] + jy) * sp.nv[2] + jz;
        const long long m = cell * ppc + sub;
        const int bz = sub % l[3], by = (sub / l[3]) % l[2], bx = (sub / (l[3] * l[2])) % l[1];
        const int a = sub / (l[3] * l[2] * l[1]);
        const int j[3] = {jx, jy, jz}, b[3] = {bx, by, bz};
        MarkerIn3 o;
        const double J0 = (jitter_u01(seed, s, m, 0) - 0.5) * jitter;
        o.xi = (double)i + ((double)a + 0.5 + J0) / l[0];
        for (int d = 0; d < 3; ++d) {
            const double Jd = (jitter_u01(seed, s, m, d + 1) - 0.5) * jitter;
            o.v[d] = sp.vmin[d] + ((double)j[d] + ((double)b[d] + 0.5 + Jd) / l[d + 1]) * sp.dv[d];
        }
        o.f = f0_value(f0, 3, sp.nx * sp.dx, o.xi * sp.dx, o.v);
        o.ok = true;
        return o;
    }
};

struct ArraySrc3 {
    const double* x;
    const double* v;   // component-major: v[d * n + k]
    const double* f;
    long long n;
    __device__ MarkerIn3 get(const SpDev& sp, long long k) const
    {
        MarkerIn3 o;
        const double L = sp.nx * sp.dx;
        const double xv = x[k];
        o.f = f[k];
        o.ok = (xv >= 0.0 && xv < L) && isfinite(o.f);
        for (int d = 0; d < 3; ++d) {
            o.v[d] = v[(long long)d * n + k];
            o.ok = o.ok && isfinite(o.v[d]);
        }
        o.xi = o.ok ? xv / sp.dx : 0.0;
        if (!o.ok) {
            for (int d = 0; d < 3; ++d) o.v[d] = sp.vmin[d];
            o.f = 0.0;
        }
        return o;
    }
};

// bucket (pencil * nkey + key) of a marker from its stored velocities
template <typename T>
__device__ __forceinline__ int bucket3(const SpDev& sp, const VCoef<T>& vc, const T (&v)[3])
{
    T w;
    const int kx = key_of(dual3(v[0], vc.a[0], vc.b[0], vc.n[0], w), vc.n[0]);
    const int ky = key_of(dual3(v[1], vc.a[1], vc.b[1], vc.n[1], w), vc.n[1]);
    const int kz = key_of(dual3(v[2], vc.a[2], vc.b[2], vc.n[2], w), vc.n[2]);
    return (kz * (vc.n[1] + 1) + ky) * sp.nkey + kx;
}

template <typename T, typename Src>
__global__ void __launch_bounds__(256) k_src3_count(const StepArgs* __restrict__ A, int s, Src src,
                                                    unsigned long long* bad)
{
    const SpDev& sp = A->sp[s];
    VCoef<T> vc;
    vc.init(sp);
    unsigned nbad = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    // whole warps iterate together (warp-aggregated counting)
    const long long n_pad = (sp.n + 31) / 32 * 32;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n_pad; k += stride) {
        const bool ok = k < sp.n;
        int b = 0;
        if (ok) {
            const MarkerIn3 mk = src.get(sp, k);
            if (!mk.ok) ++nbad;
            const T v[3] = {(T)mk.v[0], (T)mk.v[1], (T)mk.v[2]};
            b = bucket3<T>(sp, vc, v);
        }
        const int kk = ok ? b : -1;
        const unsigned grp = __match_any_sync(0xffffffffu, kk);
        if (ok && (threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(&sp.kcount[b], __popc(grp));
    }
    if (nbad && bad) atomicAdd(bad, (unsigned long long)nbad);
}

// Exclusive scan of the bucket counts over tiles of SCAN_TILE buckets (one
// block each): k_src3_tsum sums every tile, k_src3_scan adds the totals of
// the tiles before its own and scans the tile into the slot cursors kcur and
// the segment table of the target buffer, clearing the counts for the next
// use.  Creation (resort = 0) fills buffer 0; a global re-sort (resort = 1)
// fills buffer 1 - cur, and k_src3_flip makes it current after the scatter.
constexpr int SCAN_TILE = 1024;

__device__ __forceinline__ int block_sum_1024(int v, int* ws)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = __reduce_add_sync(0xffffffffu, v);
    if (lane == 0) ws[warp] = v;
    __syncthreads();
    int t = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0;
    t = __reduce_add_sync(0xffffffffu, t);
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(SCAN_TILE) k_src3_tsum(const StepArgs* __restrict__ A, int s)
{
    __shared__ int ws[32];
    const SpDev& sp = A->sp[s];
    const int nb = sp.npen * sp.nkey;
    const int i = blockIdx.x * SCAN_TILE + threadIdx.x;
    const int t = block_sum_1024(i < nb ? sp.kcount[i] : 0, ws);
    if (threadIdx.x == 0) sp.ktile[blockIdx.x] = t;
}

__global__ void __launch_bounds__(SCAN_TILE) k_src3_scan(const StepArgs* __restrict__ A, int s, int resort)
{
    __shared__ int ws[32];
    const SpDev& sp = A->sp[s];
    const int nb = sp.npen * sp.nkey, nk = sp.nkey;
    const int dst = resort ? 1 - A->ctl->cur[s] : 0;
    int o = 0;
    for (int t = threadIdx.x; t < (int)blockIdx.x; t += SCAN_TILE) o += sp.ktile[t];
    const int off = block_sum_1024(o, ws);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * SCAN_TILE + threadIdx.x;
    const int v = i < nb ? sp.kcount[i] : 0;
    int x = v;
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = ws[lane];
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += y;
        }
        ws[lane] = w;
    }
    __syncthreads();
    if (i >= nb) return;
    const int excl = off + x - v + (warp > 0 ? ws[warp - 1] : 0);
    sp.kcur[i] = excl;
    sp.kcount[i] = 0;
    int* sg = sp.seg[dst];
    const int p = i / nk, k = i - p * nk;
    sg[p * (nk + 1) + k] = excl;
    if (k == 0 && p > 0) sg[(p - 1) * (nk + 1) + nk] = excl;   // end of the previous pencil
    if (i == nb - 1) {
        sg[p * (nk + 1) + nk] = excl + v;
        if (resort && (long long)(excl + v) != sp.n) atomicOr(&A->ctl->err, ERR_CAPACITY);
    }
}

// after a global re-sort: the buffer written becomes current
__global__ void k_src3_flip(const StepArgs* __restrict__ A, int s)
{
    if (threadIdx.x == 0) {
        A->ctl->cur[s] = 1 - A->ctl->cur[s];
        A->ctl->nsort[s] += 1;
    }
}

template <typename T, typename Src>
__global__ void __launch_bounds__(256) k_src3_scatter(const StepArgs* __restrict__ A, int s, Src src)
{
    const SpDev& sp = A->sp[s];
    VCoef<T> vc;
    vc.init(sp);
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n_pad = (sp.n + 31) / 32 * 32;
    bool over = false;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n_pad; k += stride) {
        const bool ok = k < sp.n;
        MarkerIn3 mk{};
        T v[3] = {(T)0, (T)0, (T)0};
        int b = 0;
        if (ok) {
            mk = src.get(sp, k);
            for (int d = 0; d < 3; ++d) v[d] = (T)mk.v[d];
            b = bucket3<T>(sp, vc, v);
        }
        const int slot = warp_slot(sp.kcur, b, ok);
        if (!ok) continue;
        if (slot < 0 || (long long)slot >= sp.n) {
            over = true;
            continue;
        }
        const Pos3<T> pos = pos3_from_cells<T>(mk.xi, sp.nx);
        pos.store(sp, 0, slot);
        for (int d = 0; d < 3; ++d) reinterpret_cast<T*>(sp.mv[0][d])[slot] = v[d];
        reinterpret_cast<T*>(sp.mf[0])[slot] = (T)mk.f;
        if constexpr (sizeof(T) == 8) {
            double wq[4];
            marker_planes<double>(vc, v[1], v[2], wq);
            store_planes(sp.mwq[0], slot, wq);
        }
    }
    if (over) atomicOr(&A->ctl->err, ERR_CAPACITY);
}

// ---------------------------------------------------------------------------
// static background magnetic field: Boris push and global re-sort
// ---------------------------------------------------------------------------
// Boris coefficients of a species (storage precision): a = (q/m) dt / 2,
// t = a B (tangent of half the rotation angle along B), s = 2 t / (1 + |t|^2)
template <typename T>
struct BorisCoef {
    T a, t[3], s[3];
    __device__ __forceinline__ void init(const SpDev& sp, const double (&B)[3])
    {
        const double a2 = 0.5 * sp.qm_dt;
        double tt[3], t2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            tt[d] = a2 * B[d];
            t2 += tt[d] * tt[d];
        }
        const double f = 2.0 / (1.0 + t2);
        a = (T)a2;
        for (int d = 0; d < 3; ++d) {
            t[d] = (T)tt[d];
            s[d] = (T)(f * tt[d]);
        }
    }
};

// Boris push of every marker of species s in buffer cur, written back in
// place: half kick by E_x at the old position, rotation v- -> v+ about B,
// half kick, x += v_x dt.  The (pencil, key) bucket of the new velocities,
// computed from the stored values exactly as the scatter recomputes it, is
// counted into kcount (one atomic per distinct bucket of a warp).
template <typename T>
__global__ void __launch_bounds__(256) k_bpush3(const StepArgs* __restrict__ A, int s)
{
    extern __shared__ __align__(16) unsigned char smem[];
    T* Es = reinterpret_cast<T*>(smem);
    const SpDev& sp = A->sp[s];
    const int cb = A->ctl->cur[s];
    const int nx = sp.nx;
    for (int i = threadIdx.x; i < nx; i += blockDim.x)
        Es[i] = sizeof(T) == 4 ? (T)A->fd.E32[i] : (T)A->fd.E64[i];
    __syncthreads();
    BorisCoef<T> bc;
    bc.init(sp, A->fd.B);
    VCoef<T> vc;
    vc.init(sp);
    const T dt_dx = (T)sp.dt_dx;
    T* const g0 = reinterpret_cast<T*>(sp.mv[cb][0]);
    T* const g1 = reinterpret_cast<T*>(sp.mv[cb][1]);
    T* const g2 = reinterpret_cast<T*>(sp.mv[cb][2]);
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n_pad = (sp.n + 31) / 32 * 32;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n_pad; k += stride) {
        const bool ok = k < sp.n;
        int b = 0;
        if (ok) {
            Pos3<T> pos;
            pos.load(sp, cb, (int)k);
            int i0, ia, ib;
            T wx;
            pos.cic(i0, wx);
            wrap_pair(i0, nx, ia, ib);
            const T aE = bc.a * (((T)1 - wx) * Es[ia] + wx * Es[ib]);
            const T m0 = g0[k] + aE, m1 = g1[k], m2 = g2[k];
            const T p0 = m0 + (m1 * bc.t[2] - m2 * bc.t[1]);
            const T p1 = m1 + (m2 * bc.t[0] - m0 * bc.t[2]);
            const T p2 = m2 + (m0 * bc.t[1] - m1 * bc.t[0]);
            const T v[3] = {m0 + (p1 * bc.s[2] - p2 * bc.s[1]) + aE, m1 + (p2 * bc.s[0] - p0 * bc.s[2]),
                            m2 + (p0 * bc.s[1] - p1 * bc.s[0])};
            pos.drift(v[0] * dt_dx, nx);
            pos.store(sp, cb, (int)k);
            g0[k] = v[0];
            g1[k] = v[1];
            g2[k] = v[2];
            b = bucket3<T>(sp, vc, v);
        }
        const int kk = ok ? b : -1;
        const unsigned grp = __match_any_sync(0xffffffffu, kk);
        if (ok && (threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(&sp.kcount[b], __popc(grp));
    }
}

// the markers of species s from buffer cur into their (pencil, key) buckets
// of buffer 1 - cur (k_src3_scan has placed the cursors).  A warp takes
// RS3_ROUNDS x 32 consecutive markers: all loads first, then one slot per
// round (a match on the bucket and one atomic per distinct bucket, all
// rounds' atomics in flight together), then the stores.
constexpr int RS3_ROUNDS = 4;

template <typename T>
__global__ void __launch_bounds__(256) k_rs3_scatter(const StepArgs* __restrict__ A, int s)
{
    const SpDev& sp = A->sp[s];
    const int src = A->ctl->cur[s], dst = 1 - src;
    VCoef<T> vc;
    vc.init(sp);
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long n = sp.n;
    const T* f_src = reinterpret_cast<const T*>(sp.mf[src]);
    bool over = false;
    for (long long w0 = wid * 32 * RS3_ROUNDS; w0 < n; w0 += nw * 32 * RS3_ROUNDS) {
        T v[RS3_ROUNDS][3], fv[RS3_ROUNDS];
        Pos3<T> pos[RS3_ROUNDS];
        int b[RS3_ROUNDS];
#pragma unroll
        for (int r = 0; r < RS3_ROUNDS; ++r) {
            const long long k = w0 + r * 32 + lane;
            b[r] = -1;
            if (k < n) {
                for (int d = 0; d < 3; ++d) v[r][d] = reinterpret_cast<const T*>(sp.mv[src][d])[k];
                fv[r] = f_src[k];
                pos[r].load(sp, src, (int)k);
                b[r] = bucket3<T>(sp, vc, v[r]);
            }
        }
        unsigned grp[RS3_ROUNDS];
        int base[RS3_ROUNDS];
#pragma unroll
        for (int r = 0; r < RS3_ROUNDS; ++r) {
            grp[r] = __match_any_sync(0xffffffffu, b[r]);
            base[r] = 0;
            if (b[r] >= 0 && lane == __ffs(grp[r]) - 1) base[r] = atomicAdd(&sp.kcur[b[r]], __popc(grp[r]));
        }
#pragma unroll
        for (int r = 0; r < RS3_ROUNDS; ++r) {
            const int slot = __shfl_sync(0xffffffffu, base[r], __ffs(grp[r]) - 1) + __popc(grp[r] & lt);
            if (b[r] < 0) continue;
            if (slot < 0 || (long long)slot >= n) {
                over = true;
                continue;
            }
            pos[r].store(sp, dst, slot);
            for (int d = 0; d < 3; ++d) reinterpret_cast<T*>(sp.mv[dst][d])[slot] = v[r][d];
            reinterpret_cast<T*>(sp.mf[dst])[slot] = fv[r];
            if constexpr (sizeof(T) == 8) {
                double wq[4];
                marker_planes<double>(vc, v[r][1], v[r][2], wq);
                store_planes(sp.mwq[dst], slot, wq);
            }
        }
    }
    if (over) atomicOr(&A->ctl->err, ERR_CAPACITY);
}

template <typename T>
__global__ void k_get3(const StepArgs* __restrict__ A, int s, double* __restrict__ x, double* __restrict__ v,
                       double* __restrict__ f)
{
    const SpDev& sp = A->sp[s];
    const int cb = A->ctl->cur[s];
    const long long n = sp.n;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        Pos3<T> pos;
        pos.load(sp, cb, (int)k);
        if (x) x[k] = pos.cells() * sp.dx;
        if (v)
            for (int d = 0; d < 3; ++d) v[(long long)d * n + k] = (double)reinterpret_cast<const T*>(sp.mv[cb][d])[k];
        if (f) f[k] = (double)reinterpret_cast<const T*>(sp.mf[cb])[k];
    }
}

// internal [vz][vy][vx][x] -> caller [x][vx][vy][vz], 32 x 32 tiles of (x, vz)
template <typename T>
__global__ void k_getf3(const T* __restrict__ fg, const T* __restrict__ dg, int nx, int X, int Y, int Z,
                        double* __restrict__ f, double* __restrict__ n)
{
    __shared__ double tile[2][32][33];
    const int tx = (nx + 31) / 32, tz = (Z + 31) / 32;
    const long long ntile = (long long)tx * tz * X * Y;
    const long long nvf = (long long)X * Y * Z;
    for (long long t = blockIdx.x; t < ntile; t += gridDim.x) {
        const int xt = (int)(t % tx);
        long long r = t / tx;
        const int zt = (int)(r % tz);
        r /= tz;
        const int Xi = (int)(r / Y), Yi = (int)(r % Y);
        for (int rr = threadIdx.y; rr < 32; rr += blockDim.y) {
            const int zi = zt * 32 + rr, xi = xt * 32 + threadIdx.x;
            if (zi < Z && xi < nx) {
                const size_t o = (((size_t)zi * Y + Yi) * X + Xi) * nx + xi;
                tile[0][rr][threadIdx.x] = (double)fg[o];
                if (n) tile[1][rr][threadIdx.x] = (double)dg[o];
            }
        }
        __syncthreads();
        for (int rr = threadIdx.y; rr < 32; rr += blockDim.y) {
            const int xi = xt * 32 + rr, zi = zt * 32 + threadIdx.x;
            if (zi < Z && xi < nx) {
                const size_t o = (size_t)xi * nvf + ((size_t)Xi * Y + Yi) * Z + zi;
                f[o] = tile[0][threadIdx.x][rr];
                if (n) n[o] = tile[1][threadIdx.x][rr];
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static int cpt_of(int nx) { return nx <= P3_THREADS ? 1 : (nx <= 2 * P3_THREADS ? 2 : 4); }

template <typename T>
static cudaError_t set_pd3_attr(int smem)
{
    cudaError_t e;
    if ((e = raise_smem_limit(k_pd3<T, 1, false>, smem))) return e;
    if ((e = raise_smem_limit(k_pd3<T, 2, false>, smem))) return e;
    if ((e = raise_smem_limit(k_pd3<T, 4, false>, smem))) return e;
    if ((e = raise_smem_limit(k_pd3<T, 1, true>, smem))) return e;
    if ((e = raise_smem_limit(k_pd3<T, 2, true>, smem))) return e;
    return raise_smem_limit(k_pd3<T, 4, true>, smem);
}

cudaError_t configure_vhs3(const StepArgs& h)
{
    const int smem = (int)pd3_smem_bytes(h.fd.nx, nkey_max(h), h.prec);
    return h.prec == AVL_FP32 ? set_pd3_attr<float>(smem) : set_pd3_attr<double>(smem);
}

template <typename T>
static void pd3_go(const StepArgs& h, const StepArgs* d, int mode, cudaStream_t st)
{
    const int smem = (int)pd3_smem_bytes(h.fd.nx, nkey_max(h), h.prec);
    switch (cpt_of(h.fd.nx)) {
        case 1:
            if (mode == 1) k_pd3<T, 1, true><<<h.npen_total, P3_THREADS, smem, st>>>(d, mode);
            else k_pd3<T, 1, false><<<h.npen_total, P3_THREADS, smem, st>>>(d, mode);
            break;
        case 2:
            if (mode == 1) k_pd3<T, 2, true><<<h.npen_total, P3_THREADS, smem, st>>>(d, mode);
            else k_pd3<T, 2, false><<<h.npen_total, P3_THREADS, smem, st>>>(d, mode);
            break;
        default:
            if (mode == 1) k_pd3<T, 4, true><<<h.npen_total, P3_THREADS, smem, st>>>(d, mode);
            else k_pd3<T, 4, false><<<h.npen_total, P3_THREADS, smem, st>>>(d, mode);
            break;
    }
}

cudaError_t launch_pd3(const StepArgs& h, const StepArgs* d, int mode, cudaStream_t st)
{
    if (h.npen_total == 0) return cudaSuccess;
    if (h.prec == AVL_FP32)
        pd3_go<float>(h, d, mode, st);
    else
        pd3_go<double>(h, d, mode, st);
    return cudaGetLastError();
}

cudaError_t launch_fin3(const StepArgs& h, const StepArgs* d, int all_species, cudaStream_t st)
{
    if (h.prec == AVL_FP32)
        k_fin3<float><<<h.nfin_total, FIN3_X * FIN3_R, 0, st>>>(d, all_species);
    else
        k_fin3<double><<<h.nfin_total, FIN3_X * FIN3_R, 0, st>>>(d, all_species);
    return cudaGetLastError();
}

cudaError_t launch_sort3(const StepArgs& h, const StepArgs* d, cudaStream_t st)
{
    if (h.npen_total == 0) return cudaSuccess;
    if (h.prec == AVL_FP32)
        k_sort3<float><<<h.npen_total, P3_THREADS, 0, st>>>(d);
    else
        k_sort3<double><<<h.npen_total, P3_THREADS, 0, st>>>(d);
    return cudaGetLastError();
}

// bucket counts -> cursors and segment table (creation: buffer 0; re-sort:
// buffer 1 - cur)
static void scan3(const StepArgs& h, const StepArgs* d, int s, int resort, cudaStream_t st)
{
    const int nb = h.sp[s].npen * h.sp[s].nkey;
    const int tiles = (nb + SCAN_TILE - 1) / SCAN_TILE;
    k_src3_tsum<<<tiles, SCAN_TILE, 0, st>>>(d, s);
    k_src3_scan<<<tiles, SCAN_TILE, 0, st>>>(d, s, resort);
}

// source -> layout in buffer 0 (kcount is zero before and after)
template <typename Src>
static cudaError_t source_to_layout3(const StepArgs& h, const StepArgs* d, int s, Src src, unsigned long long* bad,
                                     cudaStream_t st)
{
    const long long n = h.sp[s].n;
    const int blocks = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152ll * 16));
    if (h.prec == AVL_FP32) {
        k_src3_count<float, Src><<<blocks, 256, 0, st>>>(d, s, src, bad);
        scan3(h, d, s, 0, st);
        k_src3_scatter<float, Src><<<blocks, 256, 0, st>>>(d, s, src);
    } else {
        k_src3_count<double, Src><<<blocks, 256, 0, st>>>(d, s, src, bad);
        scan3(h, d, s, 0, st);
        k_src3_scatter<double, Src><<<blocks, 256, 0, st>>>(d, s, src);
    }
    return cudaGetLastError();
}

cudaError_t launch_init3(const StepArgs& h, const StepArgs* d, int s, const int lattice[4], const avl_f0* f0_dev,
                         unsigned long long seed, double jitter, cudaStream_t st)
{
    const LatticeSrc3 src{f0_dev, seed, jitter, s, {lattice[0], lattice[1], lattice[2], lattice[3]}};
    return source_to_layout3(h, d, s, src, nullptr, st);
}

cudaError_t launch_set3(const StepArgs& h, const StepArgs* d, int s, long long n, const double* x, const double* v,
                        const double* f, unsigned long long* bad, cudaStream_t st)
{
    const ArraySrc3 src{x, v, f, n};
    return source_to_layout3(h, d, s, src, bad, st);
}

static int marker_blocks(long long n)
{
    return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152ll * 16));
}

cudaError_t launch_bpush3(const StepArgs& h, const StepArgs* d, int s, cudaStream_t st)
{
    const long long n = h.sp[s].n;
    if (n == 0) return cudaSuccess;
    const int blocks = marker_blocks(n);
    if (h.prec == AVL_FP32)
        k_bpush3<float><<<blocks, 256, (size_t)h.sp[s].nx * 4, st>>>(d, s);
    else
        k_bpush3<double><<<blocks, 256, (size_t)h.sp[s].nx * 8, st>>>(d, s);
    return cudaGetLastError();
}

cudaError_t launch_rsort3(const StepArgs& h, const StepArgs* d, int s, cudaStream_t st)
{
    const long long n = h.sp[s].n;
    if (n == 0) return cudaSuccess;
    const int blocks = marker_blocks(n);
    scan3(h, d, s, 1, st);
    if (h.prec == AVL_FP32)
        k_rs3_scatter<float><<<blocks, 256, 0, st>>>(d, s);
    else
        k_rs3_scatter<double><<<blocks, 256, 0, st>>>(d, s);
    k_src3_flip<<<1, 32, 0, st>>>(d, s);
    return cudaGetLastError();
}

cudaError_t launch_get3(const StepArgs& h, const StepArgs* d, int s, double* x, double* v, double* f, cudaStream_t st)
{
    const long long n = h.sp[s].n;
    if (n == 0) return cudaSuccess;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 152ll * 16);
    if (h.prec == AVL_FP32)
        k_get3<float><<<blocks, 256, 0, st>>>(d, s, x, v, f);
    else
        k_get3<double><<<blocks, 256, 0, st>>>(d, s, x, v, f);
    return cudaGetLastError();
}

cudaError_t launch_getf3(const StepArgs& h, int s, int which, double* f, double* n, cudaStream_t st)
{
    const SpDev& sp = h.sp[s];
    const size_t cells = (size_t)sp.nvflat * sp.nx;
    const long long ntile = (long long)((sp.nx + 31) / 32) * ((sp.nv[2] + 31) / 32) * sp.nv[0] * sp.nv[1];
    const int blocks = (int)std::max<long long>(1, std::min<long long>(ntile, 152ll * 32));
    dim3 block(32, 8);
    if (h.prec == AVL_FP32) {
        const float* dg = reinterpret_cast<const float*>(sp.acc[which]) + cells;
        k_getf3<float><<<blocks, block, 0, st>>>(reinterpret_cast<const float*>(sp.fgrid), dg, sp.nx, sp.nv[0],
                                                 sp.nv[1], sp.nv[2], f, n);
    } else {
        const double* dg = reinterpret_cast<const double*>(sp.acc[which]) + cells;
        k_getf3<double><<<blocks, block, 0, st>>>(reinterpret_cast<const double*>(sp.fgrid), dg, sp.nx, sp.nv[0],
                                                  sp.nv[1], sp.nv[2], f, n);
    }
    return cudaGetLastError();
}

}  // namespace avl
