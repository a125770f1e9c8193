// k_adjoint.cu -- discrete adjoint of the 1d1v time step on the GPU.
//
// Objective: J = 1/2 sum_i E_i(T)^2 dx after nsteps steps (the field energy
// of Eq. 12 with the factor 1/2 and no 1/cP).  Parameters: the mode
// amplitudes and beam x-drifts of the initial distribution f0 of one species
// (Sec. 3.3 / Eq. 17 form); they enter only through the marker values
// f_l = f0(x_l, v_l), so dJ/dtheta = sum_l mu_l df0_l/dtheta with
// mu_l = dJ/df_l, the total derivative through every later reconstruction
// (Eq. 4), moment (Eq. 14), Poisson solve (Eq. 6) and push (Sec. 2).
//
// The engine keeps its own markers in the fixed lattice order (marker m =
// cell * ppc + sub, as created), so that the adjoint variables of a marker
// stay aligned across steps.  Per step n the forward pass deposits with
// global atomics, forms F = N / D and the charge, solves for E (the shared
// FFT kernel) and pushes.  Checkpoints of (x, v) every K steps; the backward
// pass recomputes each segment of K states from its checkpoint, storing
// positions, velocities, the grids D, F and E of every state, then walks it
// backwards:
//   e^n   = sum_l lt_l (q/m) dt G(X^n_l),  lt = lambda_V + dt lambda_X
//           (e^N = dx E^N at the final state)
//   psi   = q dv P^T e^n = -q dv P e^n   (the multiplier of Eq. 6 is odd and
//           purely imaginary)
//   A = psi / D, B = psi F / D per cell (0 where D = 0)
//   mu   += sum_cells A alpha;  g = sum_cells (A f - B) d alpha / d(X, V)
//   lambda_X = lambda_X + lt (q/m) dt dE/dx(X^n) + g_X;  lambda_V = lt + g_V
// The cloud-in-cell derivatives are the one-sided ones of the floor() rule.
// Per-marker and per-cell arithmetic runs in the storage precision (FP64 is a
// small fraction of the FP32 rate on this GPU); mu, the charge and E stay FP64.
#include <math.h>

#include <algorithm>
#include <vector>

#include "avl_internal.cuh"
#include "common.cuh"

namespace avl {

// device-side view of the engine's buffers
struct AdjSp {
    long long n;
    int lat[2];
    unsigned long long seed;
    double jitter;
    void* hx;          // [K + 1][n] positions per slot (FP32: int cell; FP64: int64 2^-52 cells, PosX)
    float* hoff;       // [K + 1][n] FP32 offsets
    void* hv;          // [K + 1][n] velocities
    void* cx;          // [C][n] checkpoints
    float* coff;
    void* cv;
    void* f;           // [n] marker values
    void* lx;          // [n] lambda_X
    void* lv;          // [n] lambda_V
    double* mu;        // [n] dJ / df_l
    void* num;         // [nv][nx][2] deposit accumulator: (numerator, denominator) pairs
    void* den;         // unused
    void* hF;          // [K + 1][nv][nx] F = N / D per slot
    void* hD;          // [K + 1][nv][nx] D per slot
    void* AB;          // [nv][nx][2] grid adjoint (A, B) of the state being walked back
};

struct AdjDev {
    int ns, theta_s, K;
    int nact, act[MAXS];   // species stepped each time: mobile ones and theta_s
    int nstat, stat[MAXS]; // the others (immobile): their charge is deposited once
    AdjSp sp[MAXS];
    double* rho;       // [nx]
    double* rho_static;   // [nx] charge of the other (immobile) species, deposited once
    double* e;         // [nx] adjoint deposit
    double* tmp;       // [nx] P e
    double* hE;        // [K + 1][nx]
    double* grad;      // [nmode + nbeam] of the theta species
    const avl_f0* f0;  // [ns] (theta for theta_s)
};

template <typename T>
struct APos;
template <>
struct APos<float> {
    __device__ static Pos<float> load(const AdjSp& a, int slot, long long k)
    {
        Pos<float> p;
        p.c = reinterpret_cast<const int*>(a.hx)[(size_t)slot * a.n + k];
        p.o = a.hoff[(size_t)slot * a.n + k];
        return p;
    }
    __device__ static void store(const AdjSp& a, int slot, long long k, const Pos<float>& p)
    {
        reinterpret_cast<int*>(a.hx)[(size_t)slot * a.n + k] = p.c;
        a.hoff[(size_t)slot * a.n + k] = p.o;
    }
};
template <>
struct APos<double> {
    __device__ static PosX load(const AdjSp& a, int slot, long long k)
    {
        PosX p;
        p.X = reinterpret_cast<const long long*>(a.hx)[(size_t)slot * a.n + k];
        return p;
    }
    __device__ static void store(const AdjSp& a, int slot, long long k, const PosX& p)
    {
        reinterpret_cast<long long*>(a.hx)[(size_t)slot * a.n + k] = p.X;
    }
};

// velocity dual row j0 and weight w of row j0 + 1 (t = (v - vmin)/dv - 1/2),
// in the storage precision with one explicit fused multiply-add, so that
// the deposit and the gather find the same row and weight
template <typename T>
__device__ __forceinline__ int vrow(T v, const SpDev& sp, T& w)
{
    const T a = (T)sp.inv_dv[0], b = (T)(-sp.vmin[0] * sp.inv_dv[0] - 0.5);
    T t;
    if constexpr (sizeof(T) == 4)
        t = __fmaf_rn(v, a, b);
    else
        t = __fma_rn(v, a, b);
    if (!(t > (T)-2 && t < (T)(sp.nv[0] + 1))) {
        w = (T)0;
        return t > (T)0 ? sp.nv[0] + 1 : -2;
    }
    const T fl = floor(t);
    w = t - fl;
    return (int)fl;
}

// (numerator, denominator) of one cell in one reduction: a v2 FP32
// reduction in the FP32 path, two FP64 ones in the FP64 path
__device__ __forceinline__ void pair_add(float* p, float n, float d)
{
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(n), "f"(d) : "memory");
}
__device__ __forceinline__ void pair_add(double* p, double n, double d)
{
    atomicAdd(p, n);
    atomicAdd(p + 1, d);
}

// lattice marker m (order m = (i nv + j) ppc + a pv + b) of species s
template <typename T>
__global__ void k_ad_init(const StepArgs* __restrict__ A, const AdjDev* __restrict__ D, int s)
{
    const SpDev& sp = A->sp[s];
    const AdjSp& a = D->sp[s];
    const avl_f0* f0 = D->f0 + s;
    const int px = a.lat[0], pv = a.lat[1], ppc = px * pv;
    for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < a.n; m += (long long)gridDim.x * blockDim.x) {
        const long long cell = m / ppc;
        const int sub = (int)(m - cell * ppc);
        const int i = (int)(cell / sp.nv[0]), j = (int)(cell - (long long)i * sp.nv[0]);
        const int ia = sub / pv, ib = sub - ia * pv;
        const double J0 = (jitter_u01(a.seed, s, m, 0) - 0.5) * a.jitter;
        const double J1 = (jitter_u01(a.seed, s, m, 1) - 0.5) * a.jitter;
        const double xi = (double)i + ((double)ia + 0.5 + J0) / px;
        const double v[3] = {sp.vmin[0] + ((double)j + ((double)ib + 0.5 + J1) / pv) * sp.dv[0], 0.0, 0.0};
        APos<T>::store(a, 0, m, posm_from_cells<T>(xi, sp.nx));
        reinterpret_cast<T*>(a.hv)[m] = (T)v[0];
        reinterpret_cast<T*>(a.f)[m] = (T)f0_value(f0, 1, sp.nx * sp.dx, xi * sp.dx, v);
        reinterpret_cast<T*>(a.lx)[m] = (T)0;
        reinterpret_cast<T*>(a.lv)[m] = (T)0;
        a.mu[m] = 0.0;
    }
}

// deposit of the markers of slot `slot` (numerator and denominator of Eq. 4)
template <typename T>
__global__ void k_ad_dep(const StepArgs* __restrict__ A, const AdjDev* __restrict__ D, int slot, int all)   // all: the static list
{
    const int s = all ? D->stat[blockIdx.y] : D->act[blockIdx.y];
    const SpDev& sp = A->sp[s];
    const AdjSp& a = D->sp[s];
    const int nx = sp.nx, nv = sp.nv[0];
    T* acc = reinterpret_cast<T*>(a.num);
    const T* f = reinterpret_cast<const T*>(a.f);
    const T* vv = reinterpret_cast<const T*>(a.hv) + (size_t)slot * a.n;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < a.n; k += (long long)gridDim.x * blockDim.x) {
        const PosM<T> p = APos<T>::load(a, slot, k);
        int i0;
        T wx;
        p.cic(i0, wx);
        int ia, ib;
        wrap_pair(i0, nx, ia, ib);
        T wv;
        const int j0 = vrow(vv[k], sp, wv);
        const T fl = f[k];
#pragma unroll
        for (int cv = 0; cv < 2; ++cv) {
            const int j = j0 + cv;
            if (j < 0 || j >= nv) continue;
            const T av = cv ? wv : (T)1 - wv;
            const T a0 = ((T)1 - wx) * av, a1 = wx * av;
            pair_add(acc + 2 * ((size_t)j * nx + ia), a0 * fl, a0);
            pair_add(acc + 2 * ((size_t)j * nx + ib), a1 * fl, a1);
        }
    }
}

// F = N / D and D into slot `slot`, accumulators cleared; charge per column
// (Eq. 14) added into rho
template <typename T>
__global__ void __launch_bounds__(256) k_ad_fin(const StepArgs* __restrict__ A, const AdjDev* __restrict__ D, int slot,
                                                int all)
{
    __shared__ double col[8][32];
    const int s = all ? D->stat[blockIdx.y] : D->act[blockIdx.y];
    const SpDev& sp = A->sp[s];
    const AdjSp& a = D->sp[s];
    const int nx = sp.nx, nv = sp.nv[0];
    const int x = blockIdx.x * 32 + (threadIdx.x & 31), lr = threadIdx.x >> 5;
    const size_t cells = (size_t)nx * nv;
    const int rg = (nv + gridDim.z - 1) / gridDim.z;   // rows of this block's group
    const int jb = blockIdx.z * rg, je = min(nv, jb + rg);
    T* acc = reinterpret_cast<T*>(a.num);
    T* F = reinterpret_cast<T*>(a.hF) + (size_t)slot * cells;
    T* Dg = reinterpret_cast<T*>(a.hD) + (size_t)slot * cells;
    double r = 0.0;
    if (x < nx) {
        for (int j = jb + lr; j < je; j += 8) {
            const size_t o = (size_t)j * nx + x;
            const T n0 = acc[2 * o], d0 = acc[2 * o + 1];
            const T fv = d0 > (T)0 ? n0 / d0 : (T)0;
            F[o] = fv;
            Dg[o] = d0;
            acc[2 * o] = (T)0;
            acc[2 * o + 1] = (T)0;
            r += (double)fv;
        }
    }
    col[lr][threadIdx.x & 31] = r;
    __syncthreads();
    if (lr == 0 && x < nx) {
        double t = 0.0;
        for (int k = 0; k < 8; ++k) t += col[k][threadIdx.x];
        atomicAdd(D->rho + x, sp.q * sp.dv[0] * t);
    }
}

// push (Sec. 2) from slot to slot + 1 with the field of slot; immobile
// species are copied
template <typename T>
__global__ void k_ad_push(const StepArgs* __restrict__ A, const AdjDev* __restrict__ D, int slot)
{
    const int s = D->act[blockIdx.y];
    const SpDev& sp = A->sp[s];
    const AdjSp& a = D->sp[s];
    const int nx = sp.nx;
    const double* E = D->hE + (size_t)slot * nx;
    const T* v0 = reinterpret_cast<const T*>(a.hv) + (size_t)slot * a.n;
    T* v1 = reinterpret_cast<T*>(a.hv) + (size_t)(slot + 1) * a.n;
    const T qm_dt = (T)sp.qm_dt, dt_dx = (T)sp.dt_dx;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < a.n; k += (long long)gridDim.x * blockDim.x) {
        PosM<T> p = APos<T>::load(a, slot, k);
        T v = v0[k];
        if (sp.mobile) {
            int i0;
            T w;
            p.cic(i0, w);
            int ia, ib;
            wrap_pair(i0, nx, ia, ib);
            const T El = ((T)1 - w) * (T)E[ia] + w * (T)E[ib];
            v = v + qm_dt * El;
            p.drift(v * dt_dx, nx);
        }
        APos<T>::store(a, slot + 1, k, p);
        v1[k] = v;
    }
}

// adjoint deposit onto the x grid: e_i += lt (q/m) dt G_i(X) over the mobile
// markers of slot (lt = lambda_V + dt lambda_X); at the final state e = dx E
// per-warp partial sums of the adjoint deposit: FP32 in the FP32 path (native
// shared-memory reductions), FP64 otherwise; one copy per warp keeps the
// contention within a warp
template <typename T>
struct EAcc {
    using type = double;
};
template <>
struct EAcc<float> {
    using type = float;
};

template <typename T>
__global__ void __launch_bounds__(256) k_ad_e(const StepArgs* __restrict__ A, const AdjDev* __restrict__ D, int slot,
                                              int terminal, int copies)
{
    using S = typename EAcc<T>::type;
    extern __shared__ __align__(16) unsigned char es_raw[];
    S* es = reinterpret_cast<S*>(es_raw);   // [8 warps][nx]
    const int s = D->act[blockIdx.y];
    const SpDev& sp = A->sp[s];
    const AdjSp& a = D->sp[s];
    const int nx = sp.nx;
    if (terminal) {
        if (blockIdx.y == 0 && blockIdx.x == 0)
            for (int i = threadIdx.x; i < nx; i += blockDim.x) D->e[i] = sp.dx * D->hE[(size_t)slot * nx + i];
        return;
    }
    if (!sp.mobile) return;
    for (int i = threadIdx.x; i < copies * nx; i += blockDim.x) es[i] = (S)0;
    __syncthreads();
    S* ew = copies ? es + ((threadIdx.x >> 5) % copies) * nx : nullptr;
    const T* lx = reinterpret_cast<const T*>(a.lx);
    const T* lv = reinterpret_cast<const T*>(a.lv);
    const T c0 = (T)sp.qm_dt;
    const T dt = (T)(sp.dt_dx * sp.dx);
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < a.n; k += (long long)gridDim.x * blockDim.x) {
        const PosM<T> p = APos<T>::load(a, slot, k);
        int i0;
        T w;
        p.cic(i0, w);
        int ia, ib;
        wrap_pair(i0, nx, ia, ib);
        const T c = (lv[k] + dt * lx[k]) * c0;
        if (copies) {
            atomicAdd(ew + ia, (S)(c * ((T)1 - w)));
            atomicAdd(ew + ib, (S)(c * w));
        } else {   // grid too large for shared copies
            atomicAdd(D->e + ia, (double)(c * ((T)1 - w)));
            atomicAdd(D->e + ib, (double)(c * w));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nx && copies; i += blockDim.x) {
        double t = 0.0;
        for (int q = 0; q < copies; ++q) t += (double)es[q * nx + i];
        if (t != 0.0) atomicAdd(D->e + i, t);
    }
}

// grid adjoint of slot: A = psi / D, B = psi F / D (0 where D = 0) with
// psi = q dv P^T e = -q dv (P e) = -q dv tmp
template <typename T>
__global__ void k_ad_grid(const StepArgs* __restrict__ A, const AdjDev* __restrict__ D, int slot)
{
    const int s = D->act[blockIdx.y];
    const SpDev& sp = A->sp[s];
    const AdjSp& a = D->sp[s];
    const int nx = sp.nx;
    const size_t cells = (size_t)nx * sp.nv[0];
    const T* F = reinterpret_cast<const T*>(a.hF) + (size_t)slot * cells;
    const T* Dg = reinterpret_cast<const T*>(a.hD) + (size_t)slot * cells;
    T* ab = reinterpret_cast<T*>(a.AB);
    const double psi_c = -sp.q * sp.dv[0];
    for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < cells; o += (size_t)gridDim.x * blockDim.x) {
        const T d = Dg[o];
        const T ps = (T)(psi_c * D->tmp[o % nx]);
        const T A_ = d > (T)0 ? ps / d : (T)0;
        ab[2 * o] = A_;
        ab[2 * o + 1] = A_ * F[o];
    }
}

// per marker: mu += sum A alpha, lambda update (see the file head)
template <typename T>
__global__ void k_ad_gather(const StepArgs* __restrict__ A, const AdjDev* __restrict__ D, int slot, int terminal)
{
    const int s = D->act[blockIdx.y];
    const SpDev& sp = A->sp[s];
    const AdjSp& a = D->sp[s];
    const int nx = sp.nx, nv = sp.nv[0];
    const T* ab = reinterpret_cast<const T*>(a.AB);
    const double* E = D->hE + (size_t)slot * nx;
    const T* vv = reinterpret_cast<const T*>(a.hv) + (size_t)slot * a.n;
    const T* f = reinterpret_cast<const T*>(a.f);
    T* lx = reinterpret_cast<T*>(a.lx);
    T* lv = reinterpret_cast<T*>(a.lv);
    const T idx_ = (T)(1.0 / sp.dx), idv = (T)sp.inv_dv[0];
    const T dt = (T)(sp.dt_dx * sp.dx);
    const T qm_dt = (T)sp.qm_dt;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < a.n; k += (long long)gridDim.x * blockDim.x) {
        const PosM<T> p = APos<T>::load(a, slot, k);
        int i0;
        T wxT;
        p.cic(i0, wxT);
        int ia, ib;
        wrap_pair(i0, nx, ia, ib);
        T wv;
        const int j0 = vrow(vv[k], sp, wv);
        const T wx = wxT, fl = f[k];
        T m = 0, gx = 0, gv = 0;
#pragma unroll
        for (int cv = 0; cv < 2; ++cv) {
            const int j = j0 + cv;
            if (j < 0 || j >= nv) continue;
            const T av = cv ? wv : (T)1 - wv, dav = cv ? idv : -idv;
#pragma unroll
            for (int cx = 0; cx < 2; ++cx) {
                const int i = cx ? ib : ia;
                const T ax = cx ? wx : (T)1 - wx, dax = cx ? idx_ : -idx_;
                const size_t o = (size_t)j * nx + i;
                const T Ac = ab[2 * o], Bc = ab[2 * o + 1];
                m += Ac * ax * av;
                const T cc = Ac * fl - Bc;
                gx += cc * dax * av;
                gv += cc * ax * dav;
            }
        }
        a.mu[k] += (double)m;
        if (terminal) {
            lx[k] = gx;
            lv[k] = gv;
        } else if (sp.mobile) {
            const T lxk = lx[k];
            const T lt = lv[k] + dt * lxk;
            const T dEdx = (T)(E[ib] - E[ia]) * idx_;
            lx[k] = lxk + lt * (qm_dt * dEdx) + gx;
            lv[k] = lt + gv;
        }
    }
}

// dJ/dtheta = sum_l mu_l df0_l/dtheta for the theta species: df0/d amp_m =
// B(v) cos(k_m x + phase_m), df0/d u_b = P(x) n_b M_b(v) (v - u_b) / vth_b^2
template <typename T>
__global__ void __launch_bounds__(256) k_ad_theta(const StepArgs* __restrict__ A, const AdjDev* __restrict__ D)
{
    const int s = D->theta_s;
    const SpDev& sp = A->sp[s];
    const AdjSp& a = D->sp[s];
    const avl_f0* f0 = D->f0 + s;
    const int nm = f0->nmode, nb = f0->nbeam, nt = nm + nb;
    __shared__ double red[64 + 4][8];
    double acc[64 + 4];
    for (int t = 0; t < nt; ++t) acc[t] = 0.0;
    const int px = a.lat[0], pv = a.lat[1], ppc = px * pv;
    const double L = sp.nx * sp.dx;
    for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < a.n; m += (long long)gridDim.x * blockDim.x) {
        const long long cell = m / ppc;
        const int sub = (int)(m - cell * ppc);
        const int i = (int)(cell / sp.nv[0]), j = (int)(cell - (long long)i * sp.nv[0]);
        const int ia = sub / pv, ib = sub - ia * pv;
        const double J0 = (jitter_u01(a.seed, s, m, 0) - 0.5) * a.jitter;
        const double J1 = (jitter_u01(a.seed, s, m, 1) - 0.5) * a.jitter;
        const double x = ((double)i + ((double)ia + 0.5 + J0) / px) * sp.dx;
        const double v = sp.vmin[0] + ((double)j + ((double)ib + 0.5 + J1) / pv) * sp.dv[0];
        const double mu = a.mu[m];
        double pert = 1.0;
        for (int q = 0; q < nm; ++q) pert += f0->amp[q] * cos(2.0 * M_PI * f0->mode[q] * x / L + f0->phase[q]);
        double B = 0.0;
        for (int b = 0; b < nb; ++b) {
            const double sd = f0->beam_vth[b][0];
            const double t = (v - f0->beam_u[b][0]) / sd;
            const double Mb = f0->beam_n[b] * exp(-0.5 * t * t) / (sqrt(2.0 * M_PI) * sd);
            B += Mb;
            acc[nm + b] += mu * pert * Mb * t / sd;
        }
        for (int q = 0; q < nm; ++q) acc[q] += mu * B * cos(2.0 * M_PI * f0->mode[q] * x / L + f0->phase[q]);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = 0; t < nt; ++t) {
        double v = acc[t];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[t][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < nt) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += red[threadIdx.x][w];
        atomicAdd(D->grad + threadIdx.x, v);
    }
}

// ---------------------------------------------------------------------------
// host: buffers and the passes
// ---------------------------------------------------------------------------
struct AdjEngine {
    int prec = -1, ns = 0, K = 0, C = 0, nx = 0;
    long long n[MAXS] = {};
    std::vector<void*> mem;
    AdjDev h{};
    AdjDev* d = nullptr;
    avl_f0* d_f0 = nullptr;
    // one full segment of K steps, forward (with pushes) and backward,
    // recorded once and replayed for every full segment
    cudaGraphExec_t g_fwd = nullptr, g_bwd = nullptr;
    int g_K = 0, g_nact = -1;
};

static cudaError_t grab(AdjEngine* E, void** p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
    if (e == cudaSuccess) E->mem.push_back(*p);
    return e;
}

static void drop_graphs(AdjEngine* E)
{
    if (E->g_fwd) cudaGraphExecDestroy(E->g_fwd);
    if (E->g_bwd) cudaGraphExecDestroy(E->g_bwd);
    E->g_fwd = E->g_bwd = nullptr;
}

void adjoint_free(AdjEngine* E)
{
    if (!E) return;
    drop_graphs(E);
    for (void* p : E->mem) cudaFree(p);
    delete E;
}

static int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152ll * 8)); }

// row groups of the finalize so that it spreads over the SMs
static int fin_groups(const AdjEngine* E)
{
    const int xb = (E->nx + 31) / 32;
    return std::max(1, std::min(64, (2 * 152 + xb - 1) / xb));
}

static long long nmax_active(const AdjEngine* E)
{
    long long nmax = 0;
    for (int k = 0; k < E->h.nact; ++k) nmax = std::max(nmax, E->n[E->h.act[k]]);
    return nmax;
}

// the Poisson solve of Eq. 6 (P rho; the backward pass applies it to e):
// the circulant product with the Green's function on many blocks where the
// context has the table, else the single-block FFT
static cudaError_t solve(const StepArgs& h, const double* in, double* out, int nx, cudaStream_t st)
{
    if (h.fd.green) return launch_poisson_dense(in, out, nx, h.fd.green, st);
    return launch_poisson(in, out, nx, h.fd.tw, h.fd.gmul, st);
}

// reconstruction of the stepped species at slot, rho = static + theirs, E
template <typename T>
static cudaError_t recon_and_field(const StepArgs& h, const StepArgs* dA, AdjEngine* E, int slot, cudaStream_t st)
{
    cudaError_t e = cudaMemcpyAsync(E->h.rho, E->h.rho_static, (size_t)E->nx * 8, cudaMemcpyDeviceToDevice, st);
    if (e) return e;
    k_ad_dep<T><<<dim3(grid_for(nmax_active(E)), E->h.nact), 256, 0, st>>>(dA, E->d, slot, 0);
    k_ad_fin<T><<<dim3((E->nx + 31) / 32, E->h.nact, fin_groups(E)), 256, 0, st>>>(dA, E->d, slot, 0);
    if ((e = cudaGetLastError())) return e;
    return solve(h, E->h.rho, E->h.hE + (size_t)slot * E->nx, E->nx, st);
}

// charge of the species that are not stepped (immobile, not theta): once
template <typename T>
static cudaError_t static_charge(AdjEngine* E, const StepArgs* dA, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(E->h.rho_static, 0, (size_t)E->nx * 8, st);
    if (e || E->h.nstat == 0) return e;
    long long nmax = 0;
    for (int k = 0; k < E->h.nstat; ++k) nmax = std::max(nmax, E->n[E->h.stat[k]]);
    std::swap(E->h.rho, E->h.rho_static);   // k_ad_fin adds into D->rho
    if ((e = cudaMemcpyAsync(E->d, &E->h, sizeof(AdjDev), cudaMemcpyHostToDevice, st))) return e;
    k_ad_dep<T><<<dim3(grid_for(nmax), E->h.nstat), 256, 0, st>>>(dA, E->d, 0, 1);
    k_ad_fin<T><<<dim3((E->nx + 31) / 32, E->h.nstat, fin_groups(E)), 256, 0, st>>>(dA, E->d, 0, 1);
    if ((e = cudaGetLastError())) return e;
    std::swap(E->h.rho, E->h.rho_static);
    return cudaMemcpyAsync(E->d, &E->h, sizeof(AdjDev), cudaMemcpyHostToDevice, st);
}

template <typename T>
static cudaError_t push_slot(AdjEngine* E, const StepArgs* dA, int slot, cudaStream_t st)
{
    k_ad_push<T><<<dim3(grid_for(nmax_active(E)), E->h.nact), 256, 0, st>>>(dA, E->d, slot);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t back_step(const StepArgs& h, const StepArgs* dA, AdjEngine* E, int slot, int terminal, cudaStream_t st)
{
    const long long nmax = nmax_active(E);
    cudaError_t e = cudaMemsetAsync(E->h.e, 0, (size_t)E->nx * 8, st);
    if (e) return e;
    const size_t copy_bytes = (size_t)E->nx * sizeof(typename EAcc<T>::type);
    const int copies = (int)std::min<size_t>(8, (48 * 1024) / copy_bytes);
    k_ad_e<T><<<dim3(grid_for(nmax), E->h.nact), 256, copies * copy_bytes, st>>>(dA, E->d, slot, terminal, copies);
    if ((e = cudaGetLastError())) return e;
    if ((e = solve(h, E->h.e, E->h.tmp, E->nx, st))) return e;
    k_ad_grid<T><<<dim3(152 * 2, E->h.nact), 256, 0, st>>>(dA, E->d, slot);
    k_ad_gather<T><<<dim3(grid_for(nmax), E->h.nact), 256, 0, st>>>(dA, E->d, slot, terminal);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t fwd_segment(const StepArgs& h, const StepArgs* dA, AdjEngine* E, int len, bool push_last,
                               cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < len && !e; ++j) {
        e = recon_and_field<T>(h, dA, E, j, st);
        if (!e && (push_last || j + 1 < len)) e = push_slot<T>(E, dA, j, st);
    }
    return e;
}

template <typename T>
static cudaError_t bwd_segment(const StepArgs& h, const StepArgs* dA, AdjEngine* E, int len, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    for (int j = len - 1; j >= 0 && !e; --j) e = back_step<T>(h, dA, E, j, 0, st);
    return e;
}

// record `body` (launches on st) as a graph and instantiate it
template <typename F>
static cudaError_t record(cudaStream_t st, cudaGraphExec_t* out, F body)
{
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e) return e;
    cudaError_t eb = body();
    e = cudaStreamEndCapture(st, &g);
    if (eb || e) {
        if (g) cudaGraphDestroy(g);
        return eb ? eb : e;
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return e;
}

// full segments replay the recorded graphs (kernel attributes are set by a
// first direct launch before any recording)
template <typename T>
static cudaError_t full_fwd(const StepArgs& h, const StepArgs* dA, AdjEngine* E, bool push_last, cudaStream_t st)
{
    const int K = E->K;
    if (!push_last) return fwd_segment<T>(h, dA, E, K, false, st);
    if (!E->g_fwd) {
        cudaError_t e = record(st, &E->g_fwd, [&] { return fwd_segment<T>(h, dA, E, K, true, st); });
        if (e) return e;
    }
    return cudaGraphLaunch(E->g_fwd, st);
}

template <typename T>
static cudaError_t full_bwd(const StepArgs& h, const StepArgs* dA, AdjEngine* E, cudaStream_t st)
{
    if (!E->g_bwd) {
        cudaError_t e = record(st, &E->g_bwd, [&] { return bwd_segment<T>(h, dA, E, E->K, st); });
        if (e) return e;
    }
    return cudaGraphLaunch(E->g_bwd, st);
}

// copy the state of slot a (positions, velocities) of every species into the
// checkpoint c (to_ckpt) or back from it into slot a
static cudaError_t ckpt_copy(AdjEngine* E, int c, int a, bool to_ckpt, cudaStream_t st)
{
    const size_t pb = E->prec == AVL_FP32 ? 4 : 8;
    for (int s = 0; s < E->ns; ++s) {
        const AdjSp& q = E->h.sp[s];
        const size_t n = (size_t)q.n;
        auto cp = [&](void* ck, void* hs, size_t eb) {
            char* cptr = static_cast<char*>(ck) + (size_t)c * n * eb;
            char* hptr = static_cast<char*>(hs) + (size_t)a * n * eb;
            return to_ckpt ? cudaMemcpyAsync(cptr, hptr, n * eb, cudaMemcpyDeviceToDevice, st)
                           : cudaMemcpyAsync(hptr, cptr, n * eb, cudaMemcpyDeviceToDevice, st);
        };
        cudaError_t e = cp(q.cx, q.hx, pb);
        if (!e && E->prec == AVL_FP32) e = cp(q.coff, q.hoff, 4);
        if (!e) e = cp(q.cv, q.hv, pb);
        if (e) return e;
    }
    return cudaSuccess;
}

template <typename T>
static cudaError_t run(const StepArgs& h, const StepArgs* dA, AdjEngine* E, int nsteps, cudaStream_t st,
                       double* grad_host, int ngrad, double* J)
{
    cudaError_t e;
    const int K = E->K;
    if (E->g_K != K || E->g_nact != E->h.nact) {
        drop_graphs(E);
        E->g_K = K;
        E->g_nact = E->h.nact;
    }
    // initial state into slot 0
    for (int s = 0; s < E->ns; ++s) {
        k_ad_init<T><<<grid_for(E->n[s]), 256, 0, st>>>(dA, E->d, s);
        if ((e = cudaGetLastError())) return e;
    }
    if ((e = static_charge<T>(E, dA, st))) return e;
    if ((e = cudaMemsetAsync(E->h.grad, 0, 8 * (64 + 4), st))) return e;
    // forward: segments of K steps; checkpoint c = state c K
    const int nseg = std::max(1, (nsteps + K - 1) / K);
    int last_len = nsteps;
    for (int c = 0; c < nseg; ++c) {
        const int len = std::min(K, nsteps - c * K);
        if ((e = ckpt_copy(E, c, 0, true, st))) return e;
        if (len == K && c > 0) {
            if ((e = full_fwd<T>(h, dA, E, true, st))) return e;
        } else if ((e = fwd_segment<T>(h, dA, E, len, true, st))) {
            return e;
        }
        last_len = len;
        if (c + 1 < nseg && (e = ckpt_copy(E, c + 1, len, true, st))) return e;
        if (c + 1 < nseg && (e = ckpt_copy(E, c + 1, 0, false, st))) return e;
    }
    if (nsteps == 0) last_len = 0;
    // final state: its field and J, then the backward walk of the last segment
    if ((e = recon_and_field<T>(h, dA, E, last_len, st))) return e;
    std::vector<double> Ef(E->nx);
    if ((e = cudaMemcpyAsync(Ef.data(), E->h.hE + (size_t)last_len * E->nx, E->nx * 8, cudaMemcpyDeviceToHost, st)))
        return e;
    if ((e = back_step<T>(h, dA, E, last_len, 1, st))) return e;
    if ((e = bwd_segment<T>(h, dA, E, last_len, st))) return e;
    // earlier segments: recompute from the checkpoint, then walk back
    for (int c = nseg - 2; c >= 0; --c) {
        if ((e = ckpt_copy(E, c, 0, false, st))) return e;
        if ((e = full_fwd<T>(h, dA, E, true, st))) return e;
        if ((e = full_bwd<T>(h, dA, E, st))) return e;
    }
    k_ad_theta<T><<<grid_for(E->n[E->h.theta_s]), 256, 0, st>>>(dA, E->d);
    if ((e = cudaGetLastError())) return e;
    if ((e = cudaMemcpyAsync(grad_host, E->h.grad, ngrad * 8, cudaMemcpyDeviceToHost, st))) return e;
    if ((e = cudaStreamSynchronize(st))) return e;
    double s2 = 0.0;
    for (int i = 0; i < E->nx; ++i) s2 += Ef[i] * Ef[i];
    *J = 0.5 * s2 * h.fd.dx;
    return cudaSuccess;
}

cudaError_t adjoint_run(AdjEngine** eng, const StepArgs& h, const StepArgs* dA, const AdjSpec& spec, cudaStream_t st,
                        double* dJ_amp, double* dJ_u, double* J)
{
    const int ns = h.ns, nx = h.fd.nx;
    const int K = std::max(1, std::min(spec.ckpt_every, std::max(1, spec.nsteps)));
    const int C = std::max(1, (spec.nsteps + K - 1) / K);
    const size_t pb = h.prec == AVL_FP32 ? 4 : 8;
    AdjEngine* E = *eng;
    bool fits = E && E->prec == h.prec && E->ns == ns && E->K >= K && E->C >= C && E->nx == nx;
    for (int s = 0; fits && s < ns; ++s) fits = E->n[s] == spec.n[s];
    if (!fits) {
        adjoint_free(E);
        *eng = nullptr;
        E = new AdjEngine();
        E->prec = h.prec;
        E->ns = ns;
        E->K = K;
        E->C = C;
        E->nx = nx;
        cudaError_t e = cudaSuccess;
        auto g = [&](void** p, size_t b) {
            if (!e) e = grab(E, p, b);
        };
        for (int s = 0; s < ns; ++s) {
            AdjSp& q = E->h.sp[s];
            const size_t n = (size_t)spec.n[s];
            const size_t cells = (size_t)nx * h.sp[s].nv[0];
            E->n[s] = spec.n[s];
            q.n = spec.n[s];
            g(&q.hx, (K + 1) * n * pb);
            q.hoff = nullptr;
            if (h.prec == AVL_FP32) g((void**)&q.hoff, (K + 1) * n * 4);
            g(&q.hv, (K + 1) * n * pb);
            g(&q.cx, C * n * pb);
            q.coff = nullptr;
            if (h.prec == AVL_FP32) g((void**)&q.coff, C * n * 4);
            g(&q.cv, C * n * pb);
            g(&q.f, n * pb);
            g(&q.lx, n * pb);
            g(&q.lv, n * pb);
            g((void**)&q.mu, n * 8);
            g(&q.num, 2 * cells * pb);
            q.den = nullptr;
            g(&q.AB, 2 * cells * pb);
            g(&q.hF, (K + 1) * cells * pb);
            g(&q.hD, (K + 1) * cells * pb);
            if (!e) e = cudaMemsetAsync(q.num, 0, 2 * cells * pb, st);
        }
        g((void**)&E->h.rho, nx * 8);
        g((void**)&E->h.rho_static, nx * 8);
        g((void**)&E->h.e, nx * 8);
        g((void**)&E->h.tmp, nx * 8);
        g((void**)&E->h.hE, (size_t)(K + 1) * nx * 8);
        g((void**)&E->h.grad, 8 * (64 + 4));
        g((void**)&E->d_f0, sizeof(avl_f0) * ns);
        g((void**)&E->d, sizeof(AdjDev));
        if (e) {
            adjoint_free(E);
            return e;
        }
        *eng = E;
    }
    E->h.ns = ns;
    E->h.theta_s = spec.theta_s;
    E->h.nact = 0;
    E->h.nstat = 0;
    for (int s = 0; s < ns; ++s) {
        if (h.sp[s].mobile || s == spec.theta_s)
            E->h.act[E->h.nact++] = s;
        else
            E->h.stat[E->h.nstat++] = s;
    }
    E->h.K = K;
    E->h.f0 = E->d_f0;
    for (int s = 0; s < ns; ++s) {
        AdjSp& q = E->h.sp[s];
        q.lat[0] = spec.lat[s][0];
        q.lat[1] = spec.lat[s][1];
        q.seed = spec.seed[s];
        q.jitter = spec.jitter[s];
    }
    const int saveK = E->K;
    E->K = K;
    cudaError_t e = cudaMemcpyAsync(E->d_f0, spec.f0, sizeof(avl_f0) * ns, cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(E->d, &E->h, sizeof(AdjDev), cudaMemcpyHostToDevice, st);
    if (!e) e = cudaStreamSynchronize(st);
    double grad[64 + 4] = {};
    const int nm = spec.f0[spec.theta_s].nmode, nb = spec.f0[spec.theta_s].nbeam;
    if (!e)
        e = h.prec == AVL_FP32 ? run<float>(h, dA, E, spec.nsteps, st, grad, nm + nb, J)
                               : run<double>(h, dA, E, spec.nsteps, st, grad, nm + nb, J);
    E->K = saveK;
    if (e) return e;
    for (int i = 0; i < nm; ++i) dJ_amp[i] = grad[i];
    for (int b = 0; b < nb; ++b) dJ_u[b] = grad[nm + b];
    return cudaSuccess;
}

}  // namespace avl
