// k_vhs1.cu -- 1d1v kernels of the Vlasov-Hybrid time step (Fig. 2):
//   k_pd1      gather E + push (Sec. 2) fused with the VHS deposit of the
//              numerator and denominator of Eq. 4 into a shared-memory window
//   k_fin1     f = num / den (Eq. 4), velocity moment (Eq. 14), per-block
//              diagnostics (Sec. 3.4.1)
//   k_sort*    re-binning of the markers by velocity row block
//   k_init1    lattice markers weighted to f0 (Sec. 2, Sec. 3.1)
//   k_set1 / k_get1 / k_getf  conversion to and from the caller's FP64 layout
#include <math.h>

#include <algorithm>

#include "avl_internal.cuh"
#include "ptx.cuh"

namespace avl {

// ---------------------------------------------------------------------------
// marker storage access
// ---------------------------------------------------------------------------
template <typename T>
struct Pos;

// FP32: position = int cell + FP32 offset in [0, 1)
template <>
struct Pos<float> {
    int c;
    float o;
    __device__ __forceinline__ void load(const SpDev& sp, int cb, int k)
    {
        c = reinterpret_cast<const int*>(sp.mx[cb])[k];
        o = sp.moff[cb][k];
    }
    __device__ __forceinline__ void store(const SpDev& sp, int cb, int k) const
    {
        reinterpret_cast<int*>(sp.mx[cb])[k] = c;
        sp.moff[cb][k] = o;
    }
    // cloud-in-cell: lower cell i0 (may be -1) and weight w of cell i0 + 1
    __device__ __forceinline__ void cic(int& i0, float& w) const
    {
        if (o >= 0.5f) {
            i0 = c;
            w = o - 0.5f;
        } else {
            i0 = c - 1;
            w = o + 0.5f;
        }
    }
    __device__ __forceinline__ void drift(float disp, int nx)
    {
        o += disp;
        float fo = floorf(o);
        c += static_cast<int>(fo);
        o -= fo;
        if (o >= 1.0f) {
            o -= 1.0f;
            c += 1;
        }
        if (c < 0 || c >= nx) {
            c %= nx;
            if (c < 0) c += nx;
        }
    }
};

// FP64: position in cells, xi in [0, nx)
template <>
struct Pos<double> {
    double xi;
    __device__ __forceinline__ void load(const SpDev& sp, int cb, int k)
    {
        xi = reinterpret_cast<const double*>(sp.mx[cb])[k];
    }
    __device__ __forceinline__ void store(const SpDev& sp, int cb, int k) const
    {
        reinterpret_cast<double*>(sp.mx[cb])[k] = xi;
    }
    __device__ __forceinline__ void cic(int& i0, double& w) const
    {
        double u = xi - 0.5;
        double fl = floor(u);
        i0 = static_cast<int>(fl);
        w = u - fl;
    }
    __device__ __forceinline__ void drift(double disp, int nx)
    {
        double x = xi + disp;
        double n = static_cast<double>(nx);
        if (x < 0.0 || x >= n) {
            x = fmod(x, n);
            if (x < 0.0) x += n;
            if (x >= n) x -= n;
        }
        xi = x;
    }
};

// shared-memory window accumulation of (alpha f, alpha)
__device__ __forceinline__ void acc_comp(float* hi, float* lo, float x)
{
    // compensated add: the atomic returns the old value, TwoSum recovers the
    // rounding error of old + x exactly; errors accumulate in the lo plane
    float old = atomicAdd(hi, x);
    float s = __fadd_rn(old, x);
    float bp = __fsub_rn(s, old);
    float err = __fadd_rn(__fsub_rn(old, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    if (err != 0.0f) atomicAdd(lo, err);
}

template <typename T>
struct Window;

template <>
struct Window<float> {
    // planes: num_hi, num_lo, den_hi, den_lo
    float* p;
    int plane;
    __device__ __forceinline__ void add(int cell, float a, float af)
    {
        acc_comp(p + cell, p + plane + cell, af);
        acc_comp(p + 2 * plane + cell, p + 3 * plane + cell, a);
    }
};

template <>
struct Window<double> {
    double* p;
    int plane;
    __device__ __forceinline__ void add(int cell, double a, double af)
    {
        atomicAdd(p + cell, af);
        atomicAdd(p + plane + cell, a);
    }
};

// periodic neighbours of a lower CIC cell i0 in [-1, nx-1]; clamped so that a
// non-finite position can never index outside the grid
__device__ __forceinline__ void wrap_pair(int i0, int nx, int& ia, int& ib)
{
    ia = i0 < 0 ? i0 + nx : i0;
    ib = (i0 + 1 >= nx) ? i0 + 1 - nx : i0 + 1;
    ia = min(max(ia, 0), nx - 1);
    ib = min(max(ib, 0), nx - 1);
}

__device__ __forceinline__ int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
__device__ __forceinline__ int ceil_div(int a, int b) { return a >= 0 ? (a + b - 1) / b : -((-a) / b); }

__device__ __forceinline__ int species_of(const StepArgs* A, int g, bool)
{
    int s = 0;
    while (s + 1 < A->ns && g >= A->sp[s + 1].bin_base) ++s;
    return s;
}

size_t pd1_smem_bytes(const SpDev& sp, int prec)
{
    size_t eb = (size_t)sp.nx * (prec == AVL_FP32 ? 4 : 8);
    eb = (eb + 15) & ~size_t(15);
    return eb + 32 + (size_t)16 * sp.W * sp.nx;
}

// ---------------------------------------------------------------------------
// push + deposit: one CTA per velocity bin of one species
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(PD_THREADS) k_pd1(const StepArgs* __restrict__ A, int push)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int g = blockIdx.x;
    const int s = species_of(A, g, false);
    const SpDev& sp = A->sp[s];
    if (push && !sp.mobile) return;
    Ctl* ctl = A->ctl;

    const int b = g - sp.bin_base;
    const int nx = sp.nx, tv = sp.tv, hw = sp.hw, W = sp.W, nv = sp.nv[0];
    const int cb = ctl->cur[s];
    const int beg = sp.bin_start[cb][b];
    const int end = sp.bin_start[cb][b + 1];

    size_t eb = ((size_t)nx * sizeof(T) + 15) & ~size_t(15);
    T* Es = reinterpret_cast<T*>(smem);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + eb);
    unsigned* cnt = reinterpret_cast<unsigned*>(smem + eb + 16);   // [0] dirty, [1] overflow
    unsigned char* win = smem + eb + 32;
    const int plane = W * nx;
    const size_t win_bytes = (size_t)16 * plane;

    const T* Eg = (sizeof(T) == 4) ? reinterpret_cast<const T*>(A->fd.E32)
                                   : reinterpret_cast<const T*>(A->fd.E64);
    const bool use_bulk = push && ((nx * sizeof(T)) % 16 == 0);
    if (threadIdx.x == 0) {
        cnt[0] = 0;
        cnt[1] = 0;
        if (use_bulk) {
            mbar_init(bar, 1);
            fence_mbar_init();
        }
    }
    __syncthreads();
    if (use_bulk && threadIdx.x == 0) {
        mbar_arrive_expect_tx(bar, (unsigned)(nx * sizeof(T)));
        bulk_g2s(Es, Eg, (unsigned)(nx * sizeof(T)), bar);
    }
    // zero the window while the field is in flight
    {
        float4* w4 = reinterpret_cast<float4*>(win);
        const int n4 = (int)(win_bytes / 16);
        for (int i = threadIdx.x; i < n4; i += PD_THREADS) w4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (push && !use_bulk) {
        for (int i = threadIdx.x; i < nx; i += PD_THREADS) Es[i] = Eg[i];
    }
    if (use_bulk) {
        if (!mbar_wait_bounded(bar, 0, WAIT_LIMIT)) {
            if (threadIdx.x == 0) atomicOr(&ctl->err, ERR_TIMEOUT);
            mbar_wait_bounded(bar, 0, WAIT_LIMIT);
            return;
        }
    }
    __syncthreads();

    Window<T> wacc;
    wacc.p = reinterpret_cast<T*>(win);
    wacc.plane = plane;

    const T inv_dv = (T)sp.inv_dv[0];
    const T qm_dt = (T)sp.qm_dt;
    const T dt_dx = (T)sp.dt_dx;
    const double vref = sp.vmin[0] + (double)b * tv * sp.dv[0];
    const T vref_dtdx = (T)(vref * sp.dt_dx);
    const int row_base = b * tv;
    T* dvp = reinterpret_cast<T*>(sp.mv[cb][0]);
    const T* fp = reinterpret_cast<const T*>(sp.mf[cb]);
    double* ovf_num = sp.ovf;
    double* ovf_den = sp.ovf + (size_t)sp.nvflat * nx;
    const int lane = threadIdx.x & 31;

    for (int base = beg; base < end; base += PD_THREADS * PD_UNROLL) {
        Pos<T> pos[PD_UNROLL];
        T dv[PD_UNROLL], fl[PD_UNROLL];
#pragma unroll
        for (int u = 0; u < PD_UNROLL; ++u) {
            const int k = base + u * PD_THREADS + threadIdx.x;
            if (k < end) {
                pos[u].load(sp, cb, k);
                dv[u] = dvp[k];
                fl[u] = fp[k];
            }
        }
#pragma unroll
        for (int u = 0; u < PD_UNROLL; ++u) {
            const int k = base + u * PD_THREADS + threadIdx.x;
            const bool valid = k < end;
            bool dirty = false, over = false;
            if (valid) {
                if (push) {
                    int i0, ia, ib;
                    T w;
                    pos[u].cic(i0, w);
                    wrap_pair(i0, nx, ia, ib);
                    const T El = ((T)1 - w) * Es[ia] + w * Es[ib];
                    dv[u] += qm_dt * El;
                    pos[u].drift(vref_dtdx + dv[u] * dt_dx, nx);
                    pos[u].store(sp, cb, k);
                    dvp[k] = dv[u];
                }
                // deposit at the new position (Eq. 4 numerator and denominator)
                int i0, ia, ib;
                T wx;
                pos[u].cic(i0, wx);
                wrap_pair(i0, nx, ia, ib);
                const T t = dv[u] * inv_dv - (T)0.5;
                const T ft = floor(t);
                const int r0 = (int)ft;
                const T wv = t - ft;
                const T a00 = ((T)1 - wx) * ((T)1 - wv), a10 = wx * ((T)1 - wv);
                const T a01 = ((T)1 - wx) * wv, a11 = wx * wv;
                const int wr = r0 + hw;
                if (wr >= 0 && wr + 1 < W) {
                    const int c0 = wr * nx;
                    wacc.add(c0 + ia, a00, a00 * fl[u]);
                    wacc.add(c0 + ib, a10, a10 * fl[u]);
                    wacc.add(c0 + nx + ia, a01, a01 * fl[u]);
                    wacc.add(c0 + nx + ib, a11, a11 * fl[u]);
                } else {
                    const int j0 = row_base + r0;
                    if (j0 >= 0 && j0 < nv) {
                        over = true;
                        atomicAdd(ovf_num + (size_t)j0 * nx + ia, (double)(a00 * fl[u]));
                        atomicAdd(ovf_den + (size_t)j0 * nx + ia, (double)a00);
                        atomicAdd(ovf_num + (size_t)j0 * nx + ib, (double)(a10 * fl[u]));
                        atomicAdd(ovf_den + (size_t)j0 * nx + ib, (double)a10);
                    }
                    if (j0 + 1 >= 0 && j0 + 1 < nv) {
                        over = true;
                        atomicAdd(ovf_num + (size_t)(j0 + 1) * nx + ia, (double)(a01 * fl[u]));
                        atomicAdd(ovf_den + (size_t)(j0 + 1) * nx + ia, (double)a01);
                        atomicAdd(ovf_num + (size_t)(j0 + 1) * nx + ib, (double)(a11 * fl[u]));
                        atomicAdd(ovf_den + (size_t)(j0 + 1) * nx + ib, (double)a11);
                    }
                }
                // has the marker wandered out of its bin (re-sort trigger)?
                int row = row_base + (int)floor(dv[u] * inv_dv);
                row = row < 0 ? 0 : (row >= nv ? nv - 1 : row);
                dirty = (row < row_base - sp.hd) || (row >= row_base + tv + sp.hd);
            }
            const unsigned bd = __ballot_sync(0xffffffffu, dirty);
            const unsigned bo = __ballot_sync(0xffffffffu, over);
            if (lane == 0 && (bd | bo)) {
                if (bd) atomicAdd(&cnt[0], (unsigned)__popc(bd));
                if (bo) atomicAdd(&cnt[1], (unsigned)__popc(bo));
            }
        }
    }
    __syncthreads();
    // flush the window to this bin's partial sums with one bulk copy
    if (threadIdx.x == 0) {
        fence_proxy_async_smem();
        unsigned char* dst = reinterpret_cast<unsigned char*>(sp.partial) + (size_t)b * win_bytes;
        bulk_s2g(dst, win, (unsigned)win_bytes);
        bulk_commit();
        if (cnt[0]) atomicAdd(&ctl->dirty[s], (unsigned long long)cnt[0]);
        if (cnt[1]) atomicAdd(&ctl->ovf_count[s], (unsigned long long)cnt[1]);
        bulk_wait_all();
    }
}

// ---------------------------------------------------------------------------
// finalize: f = num / den (Eq. 4), charge per row group (Eq. 14), diagnostics
// ---------------------------------------------------------------------------
// FP32 path: float-float arithmetic (an unevaluated sum hi + lo) so that the
// cell values and the column sums keep the accuracy of the compensated
// deposit without per-cell FP64 work.
struct ff {
    float hi, lo;
};

__device__ __forceinline__ void ff_add(ff& a, float x)
{
    const float s = __fadd_rn(a.hi, x);
    const float bp = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    a.hi = s;
    a.lo = __fadd_rn(a.lo, e);
}

template <typename T>
struct CellSum;

template <>
struct CellSum<float> {
    ff num{0.f, 0.f}, den{0.f, 0.f};
    __device__ __forceinline__ void add_partial(const float* p, int plane)
    {
        ff_add(num, p[0]);
        num.lo = __fadd_rn(num.lo, p[plane]);
        ff_add(den, p[2 * plane]);
        den.lo = __fadd_rn(den.lo, p[3 * plane]);
    }
    __device__ __forceinline__ void add_ovf(double n, double d)
    {
        ff_add(num, (float)n);
        num.lo = __fadd_rn(num.lo, (float)(n - (double)(float)n));
        ff_add(den, (float)d);
        den.lo = __fadd_rn(den.lo, (float)(d - (double)(float)d));
    }
    // f = num / den as float-float (q, r / den); den = 0 gives f = 0
    __device__ __forceinline__ void value(float& fh, float& fl, float& dsum) const
    {
        dsum = __fadd_rn(den.hi, den.lo);
        if (den.hi > 0.f) {
            const float q = __fdiv_rn(num.hi, den.hi);
            float r = fmaf(-q, den.hi, num.hi);
            r = __fadd_rn(r, __fsub_rn(num.lo, __fmul_rn(q, den.lo)));
            fh = q;
            fl = __fdiv_rn(r, den.hi);
        } else {
            fh = 0.f;
            fl = 0.f;
        }
    }
};

template <>
struct CellSum<double> {
    double num = 0.0, den = 0.0;
    __device__ __forceinline__ void add_partial(const double* p, int plane)
    {
        num += p[0];
        den += p[plane];
    }
    __device__ __forceinline__ void add_ovf(double n, double d)
    {
        num += n;
        den += d;
    }
    __device__ __forceinline__ void value(double& fh, double& fl, double& dsum) const
    {
        dsum = den;
        fh = den > 0.0 ? num / den : 0.0;
        fl = 0.0;
    }
};

template <typename T>
struct ColAcc;

template <>
struct ColAcc<float> {
    ff rho{0.f, 0.f}, w{0.f, 0.f}, ent{0.f, 0.f};
    __device__ __forceinline__ void add(float fh, float fl, float v2)
    {
        ff_add(rho, fh);
        rho.lo = __fadd_rn(rho.lo, fl);
        ff_add(w, __fmul_rn(v2, fh));
        if (fh > 0.f) ff_add(ent, __fmul_rn(fh, logf(fh)));
    }
    __device__ __forceinline__ double r() const { return (double)rho.hi + (double)rho.lo; }
    __device__ __forceinline__ double wk() const { return (double)w.hi + (double)w.lo; }
    __device__ __forceinline__ double s() const { return (double)ent.hi + (double)ent.lo; }
};

template <>
struct ColAcc<double> {
    double rho = 0.0, w = 0.0, ent = 0.0;
    __device__ __forceinline__ void add(double fh, double, double v2)
    {
        rho += fh;
        w += v2 * fh;
        if (fh > 0.0) ent += fh * log(fh);
    }
    __device__ __forceinline__ double r() const { return rho; }
    __device__ __forceinline__ double wk() const { return w; }
    __device__ __forceinline__ double s() const { return ent; }
};

__device__ __forceinline__ int species_of_fin(const StepArgs* A, int g)
{
    int s = 0;
    while (s + 1 < A->ns && g >= A->sp[s + 1].fin_base) ++s;
    return s;
}

template <typename T>
__global__ void __launch_bounds__(FIN_THREADS) k_fin1(const StepArgs* __restrict__ A, int all_species)
{
    constexpr int RL = FIN_THREADS / FIN_XB;   // row lanes
    __shared__ double col_red[RL][FIN_XB];
    __shared__ double red[3][FIN_THREADS / 32];
    const int g = blockIdx.x;
    const int s = species_of_fin(A, g);
    const SpDev& sp = A->sp[s];
    if (!all_species && !sp.mobile) return;
    Ctl* ctl = A->ctl;
    const int blk = g - sp.fin_base;
    const int xb = blk % sp.nxb, rqi = blk / sp.nxb;
    const int nx = sp.nx, nv = sp.nvflat, tv = sp.tv, hw = sp.hw, W = sp.W;
    const int col = threadIdx.x % FIN_XB, lr = threadIdx.x / FIN_XB;
    const int x = xb * FIN_XB + col;
    const bool xok = x < nx;
    const int j0 = rqi * sp.rq, j1 = min(nv, j0 + sp.rq);
    const int plane = W * nx;
    const bool any_ovf = ctl->ovf_count[s] != 0;
    double* ovf_num = sp.ovf;
    double* ovf_den = sp.ovf + (size_t)nv * nx;
    T* fg = reinterpret_cast<T*>(sp.fgrid);
    T* ng = reinterpret_cast<T*>(sp.ngrid);
    const T* part = reinterpret_cast<const T*>(sp.partial);
    const int planes = sizeof(T) == 4 ? 4 : 2;

    ColAcc<T> acc;
    if (xok) {
        for (int j = j0 + lr; j < j1; j += RL) {
            const int blo = max(ceil_div(j - tv - hw + 1, tv), 0);
            const int bhi = min(floor_div(j + hw, tv), sp.nbins - 1);
            CellSum<T> cs;
            for (int b = blo; b <= bhi; ++b) {
                const int wr = j - (b * tv - hw);
                cs.add_partial(part + (size_t)b * planes * plane + (size_t)wr * nx + x, plane);
            }
            if (any_ovf) {
                const size_t o = (size_t)j * nx + x;
                cs.add_ovf(ovf_num[o], ovf_den[o]);
                ovf_num[o] = 0.0;
                ovf_den[o] = 0.0;
            }
            T fh, fl, dsum;
            cs.value(fh, fl, dsum);
            fg[(size_t)j * nx + x] = fh + fl;
            ng[(size_t)j * nx + x] = dsum;
            const T vj = (T)(sp.vmin[0] + (j + 0.5) * sp.dv[0]);
            acc.add(fh, fl, vj * vj);
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
        double a = 0, bb = 0, c = 0;
        for (int w = 0; w < FIN_THREADS / 32; ++w) {
            a += red[0][w];
            bb += red[1][w];
            c += red[2][w];
        }
        const double cell = sp.dx * sp.dv[0];
        sp.dpart[(size_t)blk * 4 + 0] = a * cell;
        sp.dpart[(size_t)blk * 4 + 1] = 0.5 * sp.m * bb * cell;
        sp.dpart[(size_t)blk * 4 + 2] = c * cell;
        sp.dpart[(size_t)blk * 4 + 3] = 0.0;
    }
}

// ---------------------------------------------------------------------------
// re-binning: count -> scan -> scatter, only for flagged species
// ---------------------------------------------------------------------------
__device__ __forceinline__ int warp_aggregate_add(int* counters, int key)
{
    // all 32 lanes call this; key < 0 means "no slot"
    const unsigned mask = __match_any_sync(0xffffffffu, key);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    const int rank = __popc(mask & ((1u << lane) - 1u));
    int base = 0;
    if (lane == leader && key >= 0) base = atomicAdd(counters + key, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    return base + rank;
}

template <typename T>
__device__ __forceinline__ int bin_key(const SpDev& sp, int b, T dv)
{
    int row = b * sp.tv + (int)floor(dv * (T)sp.inv_dv[0]);
    row = row < 0 ? 0 : (row >= sp.nv[0] ? sp.nv[0] - 1 : row);
    return row / sp.tv;
}

template <typename T>
__global__ void __launch_bounds__(SORT_THREADS) k_sort_count1(const StepArgs* __restrict__ A)
{
    Ctl* ctl = A->ctl;
    if (!ctl->any_sort) return;
    const int g = blockIdx.x;
    const int s = species_of(A, g, false);
    if (!ctl->sort_flag[s]) return;
    const SpDev& sp = A->sp[s];
    const int b = g - sp.bin_base;
    const int cb = ctl->cur[s];
    const int beg = sp.bin_start[cb][b], end = sp.bin_start[cb][b + 1];
    const T* dvp = reinterpret_cast<const T*>(sp.mv[cb][0]);
    for (int base = beg; base < end; base += SORT_THREADS) {
        const int k = base + threadIdx.x;
        const int key = k < end ? bin_key<T>(sp, b, dvp[k]) : -1;
        warp_aggregate_add(sp.hist, key);
    }
}

__global__ void __launch_bounds__(1024) k_sort_scan(const StepArgs* __restrict__ A, int only_species)
{
    Ctl* ctl = A->ctl;
    if (only_species < 0 && !ctl->any_sort) return;
    __shared__ int warp_sums[32];
    __shared__ int carry;
    for (int s = 0; s < A->ns; ++s) {
        if (only_species >= 0 ? s != only_species : !ctl->sort_flag[s]) continue;
        const SpDev& sp = A->sp[s];
        const int nb = sp.nbins;
        // only_species >= 0: set_markers scans into the current buffer
        int* out = sp.bin_start[only_species >= 0 ? ctl->cur[s] : 1 - ctl->cur[s]];
        if (threadIdx.x == 0) carry = 0;
        __syncthreads();
        for (int base = 0; base < nb; base += 1024) {
            const int i = base + threadIdx.x;
            const int v = i < nb ? sp.hist[i] : 0;
            int x = v;
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) warp_sums[warp] = x;
            __syncthreads();
            if (warp == 0) {
                int w = warp_sums[lane];
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, w, o);
                    if (lane >= o) w += y;
                }
                warp_sums[lane] = w;
            }
            __syncthreads();
            const int incl = x + (warp > 0 ? warp_sums[warp - 1] : 0) + carry;
            if (i < nb) {
                out[i] = incl - v;
                sp.cursor[i] = incl - v;
                sp.hist[i] = 0;
            }
            __syncthreads();
            if (threadIdx.x == 1023) carry = incl;
            __syncthreads();
        }
        if (threadIdx.x == 0) out[nb] = carry;
        __syncthreads();
    }
}

template <typename T>
__device__ __forceinline__ void move_marker(const SpDev& sp, int src_buf, int k, int dst_buf, int d,
                                            T dv_shift)
{
    Pos<T> p;
    p.load(sp, src_buf, k);
    p.store(sp, dst_buf, d);
    reinterpret_cast<T*>(sp.mv[dst_buf][0])[d] = reinterpret_cast<const T*>(sp.mv[src_buf][0])[k] + dv_shift;
    reinterpret_cast<T*>(sp.mf[dst_buf])[d] = reinterpret_cast<const T*>(sp.mf[src_buf])[k];
}

template <typename T>
__global__ void __launch_bounds__(SORT_THREADS) k_scatter1(const StepArgs* __restrict__ A)
{
    Ctl* ctl = A->ctl;
    if (!ctl->any_sort) return;
    const int g = blockIdx.x;
    const int s = species_of(A, g, false);
    const SpDev& sp = A->sp[s];
    if (ctl->sort_flag[s]) {
        const int b = g - sp.bin_base;
        const int cb = ctl->cur[s];
        const int beg = sp.bin_start[cb][b], end = sp.bin_start[cb][b + 1];
        const T* dvp = reinterpret_cast<const T*>(sp.mv[cb][0]);
        for (int base = beg; base < end; base += SORT_THREADS) {
            const int k = base + threadIdx.x;
            const int key = k < end ? bin_key<T>(sp, b, dvp[k]) : -1;
            const int d = warp_aggregate_add(sp.cursor, key);
            if (key >= 0) {
                const T shift = (T)((double)(b - key) * sp.tv * sp.dv[0]);
                move_marker<T>(sp, cb, k, 1 - cb, d, shift);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned done = atomicAdd(&ctl->scatter_done, 1u);
        if (done == gridDim.x - 1) {
            __threadfence();
            for (int q = 0; q < A->ns; ++q) {
                if (ctl->sort_flag[q]) {
                    ctl->cur[q] = 1 - ctl->cur[q];
                    ctl->sort_flag[q] = 0;
                    ctl->nsort[q] += 1;
                }
            }
            ctl->any_sort = 0;
            ctl->scatter_done = 0;
            __threadfence();
        }
    }
}

// ---------------------------------------------------------------------------
// marker initialisation on a jittered lattice (Sec. 2, Sec. 3.1)
// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea & Flood 2014): output n of the generator seeded
// with `seed`.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed, unsigned long long n)
{
    unsigned long long z = seed + (n + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double jitter_u01(unsigned long long seed, int s, long long m, int d)
{
    const unsigned long long n = ((unsigned long long)(unsigned)s << 48) | ((unsigned long long)m * 4ull + d);
    return (double)(splitmix64(seed, n) >> 11) * (1.0 / 9007199254740992.0);
}

__device__ double f0_value(const avl_f0* p, int nvdim, double L, double x, const double* v)
{
    double pert = 1.0;
    for (int m = 0; m < p->nmode; ++m)
        pert += p->amp[m] * cos(2.0 * M_PI * (double)p->mode[m] / L * x + p->phase[m]);
    double sum = 0.0;
    for (int b = 0; b < p->nbeam; ++b) {
        double gb = p->beam_n[b];
        for (int d = 0; d < nvdim; ++d) {
            const double s = p->beam_vth[b][d];
            const double t = (v[d] - p->beam_u[b][d]) / s;
            gb *= exp(-0.5 * t * t) / (sqrt(2.0 * M_PI) * s);
        }
        sum += gb;
    }
    return sum * pert;
}

template <typename T>
__global__ void k_init1(const StepArgs* __restrict__ A, int s, int px, int pv, const avl_f0* __restrict__ f0,
                        unsigned long long seed, double jitter)
{
    const SpDev& sp = A->sp[s];
    const int cb = A->ctl->cur[s];
    const int nx = sp.nx, nv = sp.nv[0], tv = sp.tv;
    const int ppc = px * pv;
    const long long per_bin = (long long)tv * nx * ppc;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < sp.n;
         k += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(k / per_bin);
        const int rows = min(tv, nv - b * tv);
        const long long kl = k - (long long)b * per_bin;
        const int p = (int)(kl / ((long long)rows * nx));
        const int rem = (int)(kl - (long long)p * rows * nx);
        const int r = rem / nx;
        const int i = rem - r * nx;
        const int j = b * tv + r;
        const int a = p / pv, bv = p - a * pv;
        const long long m = ((long long)i * nv + j) * ppc + p;
        const double J0 = (jitter_u01(seed, s, m, 0) - 0.5) * jitter;
        const double J1 = (jitter_u01(seed, s, m, 1) - 0.5) * jitter;
        const double off = ((double)a + 0.5 + J0) / px;
        const double x = ((double)i + off) * sp.dx;
        const double frac_v = (double)r + ((double)bv + 0.5 + J1) / pv;   // rows above the bin base
        double v[3] = {sp.vmin[0] + ((double)j + ((double)bv + 0.5 + J1) / pv) * sp.dv[0], 0.0, 0.0};
        const double fl = f0_value(f0, 1, sp.nx * sp.dx, x, v);
        Pos<T> pos;
        if constexpr (sizeof(T) == 4) {
            pos.c = i;
            pos.o = (float)off;
            if (pos.o >= 1.0f) pos.o = 0.99999994f;
        } else {
            pos.xi = (double)i + off;
        }
        pos.store(sp, cb, (int)k);
        reinterpret_cast<T*>(sp.mv[cb][0])[k] = (T)(frac_v * sp.dv[0]);
        reinterpret_cast<T*>(sp.mf[cb])[k] = (T)fl;
    }
}

// ---------------------------------------------------------------------------
// caller markers (FP64, arbitrary order) -> binned storage
// ---------------------------------------------------------------------------
__global__ void k_set_count1(const StepArgs* __restrict__ A, int s, long long n, const double* __restrict__ x,
                             const double* __restrict__ v, const double* __restrict__ f,
                             unsigned long long* bad)
{
    const SpDev& sp = A->sp[s];
    const double L = sp.nx * sp.dx;
    for (long long base = blockIdx.x * (long long)blockDim.x; base < n; base += (long long)gridDim.x * blockDim.x) {
        const long long k = base + threadIdx.x;
        int key = -1;
        if (k < n) {
            const double xv = x[k], vv = v[k], fv = f[k];
            if (!(xv >= 0.0 && xv < L) || !isfinite(vv) || !isfinite(fv)) {
                atomicAdd(bad, 1ull);
            } else {
                int row = (int)floor((vv - sp.vmin[0]) * sp.inv_dv[0]);
                row = row < 0 ? 0 : (row >= sp.nv[0] ? sp.nv[0] - 1 : row);
                key = row / sp.tv;
            }
        }
        warp_aggregate_add(sp.hist, key);
    }
}

template <typename T>
__global__ void k_set_scatter1(const StepArgs* __restrict__ A, int s, long long n, const double* __restrict__ x,
                               const double* __restrict__ v, const double* __restrict__ f)
{
    const SpDev& sp = A->sp[s];
    const int cb = A->ctl->cur[s];
    const double L = sp.nx * sp.dx;
    for (long long base = blockIdx.x * (long long)blockDim.x; base < n; base += (long long)gridDim.x * blockDim.x) {
        const long long k = base + threadIdx.x;
        int key = -1;
        double xv = 0, vv = 0, fv = 0;
        if (k < n) {
            xv = x[k];
            vv = v[k];
            fv = f[k];
            if ((xv >= 0.0 && xv < L) && isfinite(vv) && isfinite(fv)) {   // same filter as the count
                int row = (int)floor((vv - sp.vmin[0]) * sp.inv_dv[0]);
                row = row < 0 ? 0 : (row >= sp.nv[0] ? sp.nv[0] - 1 : row);
                key = row / sp.tv;
            }
        }
        const int d = warp_aggregate_add(sp.cursor, key);
        if (key >= 0) {
            const double xi = xv / sp.dx;
            Pos<T> pos;
            if constexpr (sizeof(T) == 4) {
                double c = floor(xi);
                double o = xi - c;
                int ci = (int)c;
                if (ci >= sp.nx) {
                    ci -= sp.nx;
                }
                pos.c = ci;
                pos.o = (float)o;
                if (pos.o >= 1.0f) {
                    pos.o = 0.0f;
                    pos.c = (ci + 1) % sp.nx;
                }
            } else {
                pos.xi = xi < sp.nx ? xi : xi - sp.nx;
            }
            pos.store(sp, cb, d);
            const double vref = sp.vmin[0] + (double)key * sp.tv * sp.dv[0];
            reinterpret_cast<T*>(sp.mv[cb][0])[d] = (T)(vv - vref);
            reinterpret_cast<T*>(sp.mf[cb])[d] = (T)fv;
        }
    }
}

template <typename T>
__global__ void k_get1(const StepArgs* __restrict__ A, int s, double* __restrict__ x, double* __restrict__ v,
                       double* __restrict__ f)
{
    const SpDev& sp = A->sp[s];
    const int b = blockIdx.x;
    const int cb = A->ctl->cur[s];
    const int beg = sp.bin_start[cb][b], end = sp.bin_start[cb][b + 1];
    const double vref = sp.vmin[0] + (double)b * sp.tv * sp.dv[0];
    for (int k = beg + threadIdx.x; k < end; k += blockDim.x) {
        Pos<T> pos;
        pos.load(sp, cb, k);
        double xi;
        if constexpr (sizeof(T) == 4)
            xi = (double)pos.c + (double)pos.o;
        else
            xi = pos.xi;
        if (x) x[k] = xi * sp.dx;
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
static int max_pd_smem(const StepArgs& h)
{
    size_t m = 0;
    for (int s = 0; s < h.ns; ++s) m = std::max(m, pd1_smem_bytes(h.sp[s], h.prec));
    return (int)m;
}

// dynamic shared-memory limits, set once per context (outside any capture)
cudaError_t configure_vhs1(const StepArgs& h)
{
    const int smem = max_pd_smem(h);
    if (h.prec == AVL_FP32)
        return cudaFuncSetAttribute(k_pd1<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return cudaFuncSetAttribute(k_pd1<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t launch_pd1(const StepArgs& h, const StepArgs* d, int push, cudaStream_t st)
{
    const int smem = max_pd_smem(h);
    if (h.prec == AVL_FP32)
        k_pd1<float><<<h.nbins_total, PD_THREADS, smem, st>>>(d, push);
    else
        k_pd1<double><<<h.nbins_total, PD_THREADS, smem, st>>>(d, push);
    return cudaGetLastError();
}

cudaError_t launch_fin1(const StepArgs& h, const StepArgs* d, int all_species, cudaStream_t st)
{
    if (h.prec == AVL_FP32)
        k_fin1<float><<<h.nfin_total, FIN_THREADS, 0, st>>>(d, all_species);
    else
        k_fin1<double><<<h.nfin_total, FIN_THREADS, 0, st>>>(d, all_species);
    return cudaGetLastError();
}

cudaError_t launch_sort1(const StepArgs& h, const StepArgs* d, cudaStream_t st)
{
    if (h.prec == AVL_FP32) {
        k_sort_count1<float><<<h.nbins_total, SORT_THREADS, 0, st>>>(d);
        k_sort_scan<<<1, 1024, 0, st>>>(d, -1);
        k_scatter1<float><<<h.nbins_total, SORT_THREADS, 0, st>>>(d);
    } else {
        k_sort_count1<double><<<h.nbins_total, SORT_THREADS, 0, st>>>(d);
        k_sort_scan<<<1, 1024, 0, st>>>(d, -1);
        k_scatter1<double><<<h.nbins_total, SORT_THREADS, 0, st>>>(d);
    }
    return cudaGetLastError();
}

cudaError_t launch_init1(const StepArgs& h, const StepArgs* d, int s, const int lattice[4], const avl_f0* f0_dev,
                         unsigned long long seed, double jitter, cudaStream_t st)
{
    const long long n = h.sp[s].n;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 152LL * 16);
    if (h.prec == AVL_FP32)
        k_init1<float><<<blocks, 256, 0, st>>>(d, s, lattice[0], lattice[1], f0_dev, seed, jitter);
    else
        k_init1<double><<<blocks, 256, 0, st>>>(d, s, lattice[0], lattice[1], f0_dev, seed, jitter);
    return cudaGetLastError();
}

cudaError_t launch_set1(const StepArgs& h, const StepArgs* d, int s, long long n, const double* x, const double* v,
                        const double* f, unsigned long long* bad, cudaStream_t st)
{
    const int blocks = (int)std::min<long long>((n + 255) / 256, 152LL * 16);
    k_set_count1<<<blocks, 256, 0, st>>>(d, s, n, x, v, f, bad);
    k_sort_scan<<<1, 1024, 0, st>>>(d, s);
    if (h.prec == AVL_FP32)
        k_set_scatter1<float><<<blocks, 256, 0, st>>>(d, s, n, x, v, f);
    else
        k_set_scatter1<double><<<blocks, 256, 0, st>>>(d, s, n, x, v, f);
    return cudaGetLastError();
}

cudaError_t launch_get1(const StepArgs& h, const StepArgs* d, int s, double* x, double* v, double* f,
                        cudaStream_t st)
{
    if (h.prec == AVL_FP32)
        k_get1<float><<<h.sp[s].nbins, 256, 0, st>>>(d, s, x, v, f);
    else
        k_get1<double><<<h.sp[s].nbins, 256, 0, st>>>(d, s, x, v, f);
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
