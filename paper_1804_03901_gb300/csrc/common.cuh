// common.cuh -- device helpers shared by the 1d1v and 1d3v kernels: marker
// position storage, periodic cloud-in-cell neighbours, compensated FP32
// sums, and the marker generator (SplitMix64 jitter, analytic f0).
#pragma once
#include <math.h>

#include "avl_internal.cuh"

namespace avl {

// Raise a kernel's dynamic shared-memory limit to at least `bytes`.  The
// limit is a property of the function for the whole process, shared by every
// context, so it only ever grows (a smaller context created later must not
// lower the limit another one relies on).  Host only; call outside captures.
template <typename K>
static cudaError_t raise_smem_limit(K* kernel, int bytes)
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e) return e;
    if (fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// periodic neighbours of a lower CIC cell i0 in [-1, nx-1]; clamped so that a
// non-finite position can never index outside the grid
__device__ __forceinline__ void wrap_pair(int i0, int nx, int& ia, int& ib)
{
    ia = i0 < 0 ? i0 + nx : i0;
    ib = (i0 + 1 >= nx) ? i0 + 1 - nx : i0 + 1;
    ia = min(max(ia, 0), nx - 1);
    ib = min(max(ib, 0), nx - 1);
}

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
        const float fo = floorf(o);
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
    __device__ __forceinline__ double cells() const { return (double)c + (double)o; }
};

// FP64 marker position (step kernels and adjoint engine): a 64-bit
// fixed-point count of 2^-52 cells, x = X 2^-52 cells with
// 0 <= X < nx 2^52 < 2^63 (FP64 grids have nx < 2048).  It resolves 2^-52
// cells everywhere (a double of the same x resolves 2^-52 x), and the
// cloud-in-cell reads the weight straight from the bits: the 52 low bits of
// X - 2^51 are the mantissa of 1 + w, so that w and the lower cell cost one
// FP64 operation instead of four (the form is limited by the FP64 pipe).
// The drift converts the displacement once (a multiply and a conversion).
struct PosX {
    long long X;
    static constexpr double ONE = 4503599627370496.0;   // 2^52: one cell
    __device__ __forceinline__ void load(const SpDev& sp, int cb, int k)
    {
        X = reinterpret_cast<const long long*>(sp.mx[cb])[k];
    }
    __device__ __forceinline__ void store(const SpDev& sp, int cb, int k) const
    {
        reinterpret_cast<long long*>(sp.mx[cb])[k] = X;
    }
    // cloud-in-cell: lower cell i0 (may be -1) and weight w of cell i0 + 1
    __device__ __forceinline__ void cic(int& i0, double& w) const
    {
        const long long U = X - (1ll << 51);   // x - 1/2
        i0 = (int)(U >> 52);                   // floor (arithmetic shift)
        w = __longlong_as_double(0x3FF0000000000000ll | (U & 0x000FFFFFFFFFFFFFll)) - 1.0;
    }
    // x into [0, nx) (periodic); Y computed modulo 2^64 so that no
    // displacement overflows
    __device__ __forceinline__ void wrap(long long Y, int nx)
    {
        const long long N = (long long)nx << 52;
        if ((unsigned long long)Y >= (unsigned long long)N) {
            Y %= N;
            if (Y < 0) Y += N;
        }
        X = Y;
    }
    // displacement of `scaled` 2^-52 cells (a double, rounded to the nearest
    // count; the conversion saturates and maps NaN to 0)
    __device__ __forceinline__ void drift_scaled(double scaled, int nx)
    {
        wrap((long long)((unsigned long long)X + (unsigned long long)__double2ll_rn(scaled)), nx);
    }
    __device__ __forceinline__ void drift(double disp, int nx) { drift_scaled(disp * ONE, nx); }
    __device__ __forceinline__ double cells() const { return (double)X * (1.0 / ONE); }
    __device__ __forceinline__ static PosX from_cells(double xi, int nx)
    {
        PosX p;
        p.X = 0;
        p.drift(xi, nx);
        return p;
    }
};

template <typename T>
struct PosSel;
template <>
struct PosSel<float> {
    using type = Pos<float>;
};
template <>
struct PosSel<double> {
    using type = PosX;
};
// marker position type: FP32 int cell + FP32 offset, FP64 PosX
template <typename T>
using PosM = typename PosSel<T>::type;

// position from a value in cells (FP64) given by a caller or the generator
template <typename T>
__device__ __forceinline__ PosM<T> posm_from_cells(double xi, int nx)
{
    if constexpr (sizeof(T) == 8) {
        return PosX::from_cells(xi, nx);
    } else {
        Pos<float> p;
        const double c = floor(xi);
        int ci = (int)c;
        const double o = xi - c;
        if (ci >= nx) ci -= nx;
        if (ci < 0) ci += nx;
        p.c = min(max(ci, 0), nx - 1);
        p.o = (float)o;
        if (p.o >= 1.0f) {
            p.o = 0.0f;
            p.c = (p.c + 1) % nx;
        }
        return p;
    }
}

// ---------------------------------------------------------------------------
// compensated accumulation
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float x)
{
    const float s = __fadd_rn(hi, x);
    const float bp = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    hi = s;
    lo = __fadd_rn(lo, e);
}


// FP32 path: float-float arithmetic (an unevaluated sum hi + lo) for the sum
// of the chunks' window partials, the cell values and the column sums,
// without per-cell FP64 work.
struct ff {
    float hi, lo;
};

__device__ __forceinline__ void ff_add(ff& a, float x) { two_sum_add(a.hi, a.lo, x); }

// Natural logarithm of a positive FP64 value by table-driven argument
// reduction (P. T. P. Tang, "Table-driven implementation of the logarithm
// function in IEEE floating-point arithmetic", ACM TOMS 16, 1990): with
// f = 2^e m, m in [1, 2), and c_j = 1 + (j + 1/2) / 2048 the centre of the
// 1/2048 interval that holds m, log f = e ln 2 + log c_j + log1p(r), where
// r = m / c_j - 1 (|r| < 2^-12) and log1p(r) is its Taylor series to r^4
// (the next term is below 2e-19).  tab[j] = (log c_j, 1 / c_j), filled once
// per context (init_log_table).  Seven FP64 operations besides the exponent's
// conversion; subnormal f (found from the bits) take the library path.
__device__ __forceinline__ double log_tab(double f, const double2* __restrict__ tab)
{
    const long long b = __double_as_longlong(f);
    if (b < 0x0010000000000000ll) return log(f);
    const int e = (int)(b >> 52) - 1023;
    const int j = (int)((b >> (52 - LOG_TAB_BITS)) & (LOG_TAB_N - 1));
    const double m = __longlong_as_double((b & 0x000FFFFFFFFFFFFFll) | 0x3FF0000000000000ll);
    const double2 t = __ldg(tab + j);
    const double r = fma(m, t.y, -1.0);
    double q = fma(r, -0.25, 1.0 / 3.0);
    q = fma(r, q, -0.5);
    const double lp = fma(r * r, q, r);
    return fma((double)e, 0.69314718055994530942, t.x + lp);
}

// n / d for a normal d > 0 by one Newton-Raphson step on the reciprocal
// (r <- r + r (1 - d r), which squares its relative error) from the PTX
// approximate reciprocal (within about 2^-20), then one correction of the
// quotient (q <- q + r (n - d q)), which squares the error of q = n r again
// and leaves the rounding (P. Markstein, "Computation of elementary
// functions on the IBM RISC System/6000 processor", IBM J. Res. Dev. 34,
// 1990); other d take the division operator.
__device__ __forceinline__ double div_nr(double n, double d)
{
    const long long b = __double_as_longlong(d);
    if (b < 0x0030000000000000ll || b >= 0x7FC0000000000000ll) return n / d;   // d < 2^-1020, d >= 2^1021
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
    r = fma(r, fma(-d, r, 1.0), r);
    const double q = n * r;
    return fma(r, fma(-d, q, n), q);
}

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
    const double2* logtab = nullptr;
    __device__ __forceinline__ void add(double fh, double, double v2)
    {
        rho += fh;
        w += v2 * fh;
        if (__double_as_longlong(fh) > 0) ent += fh * log_tab(fh, logtab);   // fh > 0 (fh is not a NaN)
    }
    __device__ __forceinline__ double r() const { return rho; }
    __device__ __forceinline__ double wk() const { return w; }
    __device__ __forceinline__ double s() const { return ent; }
};

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

__device__ __forceinline__ double f0_value(const avl_f0* p, int nvdim, double L, double x, const double* v)
{
    double pert = 1.0;
    for (int m = 0; m < p->nmode; ++m)
        pert += p->amp[m] * cos(2.0 * M_PI * (double)p->mode[m] / L * x + p->phase[m]);
    double sum = 0.0;
    for (int b = 0; b < p->nbeam; ++b) {
        double gb = p->beam_n[b];
        for (int d = 0; d < nvdim; ++d) {
            const double sd = p->beam_vth[b][d];
            const double t = (v[d] - p->beam_u[b][d]) / sd;
            gb *= exp(-0.5 * t * t) / (sqrt(2.0 * M_PI) * sd);
        }
        sum += gb;
    }
    return sum * pert;
}
}  // namespace avl
