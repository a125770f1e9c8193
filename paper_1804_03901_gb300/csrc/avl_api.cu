// avl_api.cu -- host layer of the C ABI declared in include/avl.h.
//
// Owns the device state of a context, picks the binning parameters, records
// one time step (push+deposit -> finalize -> Poisson -> re-sort) as a CUDA
// graph and replays it.  All work goes to the context stream.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "avl_internal.cuh"

using namespace avl;

struct avl_ctx {
    int device = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    avl_domain dom{};
    int ns = 0;
    avl_species sp[MAXS]{};
    StepArgs h{};
    StepArgs* d_args = nullptr;
    Ctl* d_ctl = nullptr;
    avl_f0* d_f0 = nullptr;
    unsigned long long* d_bad = nullptr;
    std::vector<void*> allocs;          // context-lifetime allocations
    std::vector<void*> layout[MAXS];    // marker storage, chunk tables and partial sums per species
    int num_sms = 152;
    bool has_markers[MAXS] = {};
    void* scratch = nullptr;            // staging for caller-layout copies
    size_t scratch_bytes = 0;
    cudaGraphExec_t gexec = nullptr;
    std::string err;
    // creation parameters of each species' markers (for avl_adjoint)
    bool lattice_made[MAXS] = {};
    int lat[MAXS][4] = {};
    unsigned long long seed_s[MAXS] = {};
    double jitter_s[MAXS] = {};
    avl_f0 f0_s[MAXS] = {};
    AdjEngine* adj = nullptr;
    // marker refinement: species whose markers carry f0 of their creation, the
    // step of that creation, and the field history buffer
    bool refinable[MAXS] = {};
    long long init_step[MAXS] = {};
    void* hist_mem = nullptr;
    int force_M = 0;                    // chunk size chosen by avl_autotune (0: heuristic)
    unsigned layout_version = 0;        // bumped whenever the launch shapes change
    // a batch: independent runs advanced by one launch per kernel class
    std::vector<avl_ctx*> runs;
    avl_ctx* parent = nullptr;          // set on the runs of a batch
    void* bm_mem = nullptr;             // device BatchMap + run tables
    std::vector<unsigned> bm_versions;  // layout versions the map was built for
    int bm_pd_blocks = 0, bm_fin_blocks = 0, bm_pd_smem = 0, bm_field_smem = 0;
};

static thread_local std::string g_create_err;

namespace {

avl_status fail(avl_ctx* c, avl_status st, const std::string& msg)
{
    if (c)
        c->err = msg;
    else
        g_create_err = msg;
    return st;
}

avl_status cuda_fail(avl_ctx* c, cudaError_t e, const char* where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(c, e == cudaErrorMemoryAllocation ? AVL_ENOMEM : AVL_ECUDA, m);
}

#define AVL_CUDA(c, expr)                                    \
    do {                                                     \
        cudaError_t e_ = (expr);                             \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #expr); \
    } while (0)

cudaError_t dalloc(avl_ctx* c, void** p, size_t bytes, bool zero)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return e;
    c->allocs.push_back(*p);
    if (zero) e = cudaMemsetAsync(*p, 0, bytes, c->st);
    return e;
}

avl_status upload_args(avl_ctx* c)
{
    AVL_CUDA(c, cudaMemcpyAsync(c->d_args, &c->h, sizeof(StepArgs), cudaMemcpyHostToDevice, c->st));
    // the host copy must stay unchanged until the copy has run
    AVL_CUDA(c, cudaStreamSynchronize(c->st));
    return AVL_OK;
}

avl_status ensure_scratch(avl_ctx* c, size_t bytes)
{
    if (c->scratch_bytes >= bytes) return AVL_OK;
    if (c->scratch) {
        AVL_CUDA(c, cudaStreamSynchronize(c->st));
        cudaFree(c->scratch);
        c->scratch = nullptr;
        c->scratch_bytes = 0;
    }
    AVL_CUDA(c, cudaMalloc(&c->scratch, bytes));
    c->scratch_bytes = bytes;
    return AVL_OK;
}

int env_int(const char* name, int dflt)
{
    const char* v = getenv(name);
    return v ? atoi(v) : dflt;
}

size_t prec_bytes(int prec) { return prec == AVL_FP32 ? 4 : 8; }

void free_layout(avl_ctx* c, int s)
{
    for (void* p : c->layout[s]) cudaFree(p);
    c->layout[s].clear();
}

// Chunk layout of species s for n markers: chunk size M (a multiple of 64,
// about AVL_CHUNKS_PER_SM chunks per SM over all species), window rows Wmax
// (the rows one chunk's keys span, plus the cloud-in-cell reach and one step
// of drift on each side), marker storage (two buffers), chunk tables and
// window partial sums.  Invalidates the step graph (grid sizes change).
avl_status plan_layout(avl_ctx* c, int s, long long n)
{
    SpDev& sp = c->h.sp[s];
    // FP64 positions are fixed-point counts of 2^-52 cells (PosX): nx 2^52 < 2^63
    if (c->h.prec == AVL_FP64 && sp.nx >= 2048)
        return fail(c, AVL_EINVAL, "FP64 1d1v markers need nx < 2048");
    AVL_CUDA(c, cudaStreamSynchronize(c->st));
    free_layout(c, s);
    sp.nchunk = 0;
    sp.n = 0;
    const int per_sm = std::max(1, env_int("AVL_CHUNKS_PER_SM", 2));
    const long long target = std::max(1, per_sm * c->num_sms / c->ns);
    // small runs: chunks of at least 512 markers spread over the SMs (FP64 in
    // particular gains from the extra SMs); large runs: the target count
    long long chunks = std::min<long long>(std::max<long long>(1, (n + 511) / 512), target);
    long long M = (n + chunks - 1) / chunks;
    M = (M + 63) / 64 * 64;
    if (c->force_M > 0) M = ((long long)c->force_M + 63) / 64 * 64;
    const int m_env = env_int("AVL_CHUNK_M", 0);
    if (m_env > 0) M = (m_env + 63) / 64 * 64;
    const double mpk = std::max(1.0, (double)n / sp.nvflat);
    const int w_env = env_int("AVL_WMAX", 0);
    int Wmax = 0;
    for (;;) {
        // window: the rows one chunk's keys span, the CIC reach, a drift halo and
        // WIN_SPARE rows for the spread of a chunk's keys between re-sorts (left
        // out first when the window does not fit in shared memory); smaller
        // chunks while it still does not fit
        const int span = (int)std::ceil((double)M / mpk) + 1;
        bool fits = false;
        for (int spare = WIN_SPARE;; spare = 0) {
            Wmax = std::min(span + 2 * HALO + 1 + spare, sp.nvflat + 2 * HALO + 2);
            if (w_env > 0) Wmax = w_env;
            sp.M = (int)M;
            sp.Wmax = Wmax;
            fits = pd1_smem_bytes(sp, c->h.prec) <= 220 * 1024;
            if (fits || spare == 0) break;
        }
        if (fits || M <= 256 || w_env > 0 || m_env > 0 || c->force_M > 0) break;
        M = std::max<long long>(256, (M / 2 + 63) / 64 * 64);
    }
    const int nch = (int)((n + M - 1) / M);
    if (pd1_smem_bytes(sp, c->h.prec) > 220 * 1024)
        return fail(c, AVL_EINVAL, "window of " + std::to_string(Wmax) + " velocity rows x " + std::to_string(sp.nx) +
                                       " cells does not fit in shared memory (use fewer markers per chunk)");
    int l = 0;
    while ((1ll << l) < M) ++l;
    sp.div_l = std::max(l, 1);
    sp.div_m = (unsigned)(((1ull << (31 + sp.div_l)) + (unsigned long long)M - 1) / (unsigned long long)M);

    const size_t pb = prec_bytes(c->h.prec);
    const size_t nn = ((size_t)n + 63) / 64 * 64;
    const int nvc = c->h.nvdim;
    auto grab = [&](void** p, size_t bytes, bool zero) -> cudaError_t {
        *p = nullptr;
        cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
        if (e) return e;
        c->layout[s].push_back(*p);
        return zero ? cudaMemsetAsync(*p, 0, std::max<size_t>(bytes, 16), c->st) : cudaSuccess;
    };
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2 && !e; ++b) {
        if (!e) e = grab(&sp.mx[b], pb * nn, true);
        if (c->h.prec == AVL_FP32) {
            void* p = nullptr;
            if (!e) e = grab(&p, 4 * nn, true);
            sp.moff[b] = (float*)p;
        } else {
            sp.moff[b] = nullptr;
        }
        for (int d = 0; d < 3; ++d) {
            sp.mv[b][d] = nullptr;
            if (d < nvc && !e) e = grab(&sp.mv[b][d], pb * nn, true);
        }
        if (!e) e = grab(&sp.mf[b], pb * nn, true);
        void* kb = nullptr;
        if (!e) e = grab(&kb, (size_t)nch * 4, true);
        sp.KB[b] = (int*)kb;
    }
    void *pc0 = nullptr, *pc1 = nullptr, *po = nullptr, *pk = nullptr, *pw = nullptr;
    if (!e) e = grab(&pc0, (size_t)nch * HIST_S * 4, true);
    if (!e) e = grab(&pc1, (size_t)nch * HIST_S * 4, true);
    if (!e) e = grab(&po, (size_t)nch * HIST_S * 4, true);
    if (!e) e = grab(&pk, (size_t)nch * 4, true);
    if (!e) e = grab(&pw, (size_t)nch * 4, true);
    if (!e) e = grab(&sp.partial, (size_t)nch * window_bytes(sp, c->h.prec), true);
    if (e) {
        free_layout(c, s);
        return cuda_fail(c, e, "cudaMalloc(markers)");
    }
    sp.cnt[0] = (int*)pc0;
    sp.cnt[1] = (int*)pc1;
    sp.offs = (int*)po;
    sp.kref_tmp = (int*)pk;
    sp.wrow0 = (int*)pw;
    sp.nchunk = nch;
    sp.n = n;
    // global chunk numbering over the species
    int base = 0;
    for (int q = 0; q < c->ns; ++q) {
        c->h.sp[q].chunk_base = base;
        base += c->h.sp[q].nchunk;
    }
    c->h.nchunk_total = base;
    c->layout_version++;
    AVL_CUDA(c, configure_vhs1(c->h));
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return AVL_OK;
}

// 1d3v layout of species s for n markers: marker storage (two buffers, the
// re-sort writes the other), the segment tables of both buffers and the
// bucket counts of the creation path.  Renumbers the pencil blocks of all
// species and invalidates the step graph.
avl_status plan_layout3(avl_ctx* c, int s, long long n)
{
    SpDev& sp = c->h.sp[s];
    AVL_CUDA(c, cudaStreamSynchronize(c->st));
    free_layout(c, s);
    sp.n = 0;
    sp.npen = 0;
    const int npen = (sp.nv[1] + 1) * (sp.nv[2] + 1);
    const int nkey = sp.nv[0] + 1;
    const size_t pb = prec_bytes(c->h.prec);
    const size_t nn = ((size_t)n + 63) / 64 * 64;
    auto grab = [&](void** p, size_t bytes, bool zero) -> cudaError_t {
        *p = nullptr;
        cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
        if (e) return e;
        c->layout[s].push_back(*p);
        return zero ? cudaMemsetAsync(*p, 0, std::max<size_t>(bytes, 16), c->st) : cudaSuccess;
    };
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2 && !e; ++b) {
        e = grab(&sp.mx[b], pb * nn, true);
        sp.moff[b] = nullptr;
        if (!e && c->h.prec == AVL_FP32) {
            void* q = nullptr;
            e = grab(&q, 4 * nn, true);
            sp.moff[b] = (float*)q;
        }
        for (int d = 0; d < 3 && !e; ++d) e = grab(&sp.mv[b][d], pb * nn, true);
        if (!e) e = grab(&sp.mf[b], pb * nn, true);
        sp.mwq[b] = nullptr;
        if (!e && c->h.prec == AVL_FP64) e = grab(&sp.mwq[b], 4 * pb * nn, true);
        void* sg = nullptr;
        if (!e) e = grab(&sg, (size_t)npen * (nkey + 1) * 4, true);
        sp.seg[b] = (int*)sg;
    }
    void* kc = nullptr;
    const size_t ntile = ((size_t)npen * nkey + 1023) / 1024;
    if (!e) e = grab(&kc, (2 * (size_t)npen * nkey + ntile + 1) * 4, true);
    if (e) {
        free_layout(c, s);
        return cuda_fail(c, e, "cudaMalloc(markers)");
    }
    sp.kcount = (int*)kc;
    sp.kcur = (int*)kc + (size_t)npen * nkey;
    sp.ktile = (int*)kc + 2 * (size_t)npen * nkey;
    sp.npen = npen;
    sp.nkey = nkey;
    sp.n = n;
    int base = 0;
    for (int q = 0; q < c->ns; ++q) {
        c->h.sp[q].pen_base = base;
        base += c->h.sp[q].npen;
    }
    c->h.npen_total = base;
    c->layout_version++;
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return AVL_OK;
}

// a freshly created layout: buffer 0, key counts in buffer 0, no re-sort
// pending; the scratch counts of the creation path start at zero
avl_status set_cur_zero(avl_ctx* c, int s)
{
    const int zero = 0;
    AVL_CUDA(c, cudaMemcpyAsync(&c->d_ctl->cur[s], &zero, sizeof(int), cudaMemcpyHostToDevice, c->st));
    AVL_CUDA(c, cudaMemcpyAsync(&c->d_ctl->hsel[s], &zero, sizeof(int), cudaMemcpyHostToDevice, c->st));
    AVL_CUDA(c, cudaMemcpyAsync(&c->d_ctl->sort_now[s], &zero, sizeof(int), cudaMemcpyHostToDevice, c->st));
    AVL_CUDA(c, cudaMemcpyAsync(&c->d_ctl->sort_next[s], &zero, sizeof(int), cudaMemcpyHostToDevice, c->st));
    const SpDev& sp = c->h.sp[s];
    if (sp.nvdim == 1) {
        AVL_CUDA(c, cudaMemsetAsync(sp.far_cnt[0], 0, (size_t)sp.nvflat * 4, c->st));
        AVL_CUDA(c, cudaMemsetAsync(sp.far_cnt[1], 0, (size_t)sp.nvflat * 4, c->st));
    } else {
        const unsigned long long z = 0;
        AVL_CUDA(c, cudaMemcpyAsync(&c->d_ctl->movers[s], &z, 8, cudaMemcpyHostToDevice, c->st));
        AVL_CUDA(c, cudaMemcpyAsync(&c->d_ctl->far_movers[s], &z, 8, cudaMemcpyHostToDevice, c->st));
    }
    AVL_CUDA(c, cudaStreamSynchronize(c->st));
    return AVL_OK;
}

// before a refresh: the far-key counts of every species start at zero (the
// count kernel recounts the current state of every species with markers)
avl_status clear_far_counts(avl_ctx* c)
{
    if (c->h.nvdim == 3) return AVL_OK;
    for (int s = 0; s < c->ns; ++s) {
        const SpDev& sp = c->h.sp[s];
        AVL_CUDA(c, cudaMemsetAsync(sp.far_cnt[0], 0, (size_t)sp.nvflat * 4, c->st));
        AVL_CUDA(c, cudaMemsetAsync(sp.far_cnt[1], 0, (size_t)sp.nvflat * 4, c->st));
    }
    return AVL_OK;
}

// reconstruct every species with markers, then rho and E (no push)
avl_status refresh(avl_ctx* c)
{
    if (c->h.nvdim == 3) {
        AVL_CUDA(c, launch_pd3(c->h, c->d_args, 0, c->st));
        AVL_CUDA(c, launch_fin3(c->h, c->d_args, 1, c->st));
        AVL_CUDA(c, launch_field(c->h, c->d_args, 0, c->st));
        return AVL_OK;
    }
    avl_status st = clear_far_counts(c);
    if (st) return st;
    AVL_CUDA(c, launch_count1(c->h, c->d_args, c->st));
    // FP32 deposits sum deviations from the stored f (exact for any stored
    // values); a second pass takes the first pass's f as that reference, so
    // that a fresh marker set is reconstructed as precisely as a step
    const int passes = c->h.prec == AVL_FP32 ? 2 : 1;
    for (int p = 0; p < passes; ++p) {
        AVL_CUDA(c, launch_pd1(c->h, c->d_args, 0, c->st));
        AVL_CUDA(c, launch_fin1(c->h, c->d_args, 1, c->st));
    }
    AVL_CUDA(c, launch_field(c->h, c->d_args, 0, c->st));
    return AVL_OK;
}

// one step: push + deposit + write back (in place or re-sorted) + key counts
// of the new state -> f, rho, diagnostics -> E, and the re-sort decision and
// slots for the next step
avl_status enqueue_batch_step(avl_ctx* b);

// 1d3v with a magnetic field: Boris push of every mobile species, then the
// global (pencil, key) re-sort into the other buffer
cudaError_t launch_magnetized_push(avl_ctx* c)
{
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < c->ns && !e; ++s) {
        if (!c->h.sp[s].mobile) continue;
        e = launch_bpush3(c->h, c->d_args, s, c->st);
        if (!e) e = launch_rsort3(c->h, c->d_args, s, c->st);
    }
    return e;
}

avl_status enqueue_step(avl_ctx* c)
{
    if (!c->runs.empty()) return enqueue_batch_step(c);
    if (c->h.nvdim == 3 && c->h.fd.magnetized) {
        AVL_CUDA(c, launch_magnetized_push(c));
        AVL_CUDA(c, launch_pd3(c->h, c->d_args, 2, c->st));
        AVL_CUDA(c, launch_fin3(c->h, c->d_args, 0, c->st));
        AVL_CUDA(c, launch_field(c->h, c->d_args, 1, c->st));
        return AVL_OK;
    }
    if (c->h.nvdim == 3) {
        AVL_CUDA(c, launch_pd3(c->h, c->d_args, 1, c->st));
        AVL_CUDA(c, launch_fin3(c->h, c->d_args, 0, c->st));
        AVL_CUDA(c, launch_field(c->h, c->d_args, 1, c->st));
        AVL_CUDA(c, launch_sort3(c->h, c->d_args, c->st));
        return AVL_OK;
    }
    AVL_CUDA(c, launch_rs1(c->h, c->d_args, c->st));
    AVL_CUDA(c, launch_pd1(c->h, c->d_args, 1, c->st));
    AVL_CUDA(c, launch_fin1(c->h, c->d_args, 0, c->st));
    AVL_CUDA(c, launch_field(c->h, c->d_args, 1, c->st));
    return AVL_OK;
}

avl_status build_graph(avl_ctx* c)
{
    if (c->gexec) return AVL_OK;
    cudaGraph_t g = nullptr;
    AVL_CUDA(c, cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
    avl_status st = enqueue_step(c);
    cudaError_t e = cudaStreamEndCapture(c->st, &g);
    if (st != AVL_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&c->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->gexec = nullptr;
        return cuda_fail(c, e, "cudaGraphInstantiate");
    }
    return AVL_OK;
}

avl_status check_species(avl_ctx* c, int s)
{
    if (!c) return AVL_EINVAL;
    if (s < 0 || s >= c->ns) return fail(c, AVL_EINVAL, "species index out of range");
    return AVL_OK;
}

// the device-side error flags of the work enqueued so far; flags are cleared
// once they are reported
avl_status read_errors(avl_ctx* c)
{
    int err = 0;
    AVL_CUDA(c, cudaMemcpyAsync(&err, &c->d_ctl->err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    AVL_CUDA(c, cudaStreamSynchronize(c->st));
    if (err) {
        AVL_CUDA(c, cudaMemsetAsync(&c->d_ctl->err, 0, sizeof(int), c->st));
        AVL_CUDA(c, cudaStreamSynchronize(c->st));
    }
    if (err & ERR_TIMEOUT) return fail(c, AVL_ETIMEOUT, "a bounded device-side wait gave up");
    if (err & ERR_NUMERIC) return fail(c, AVL_ENUMERIC, "NaN or Inf in the field or diagnostics");
    if (err & ERR_CAPACITY) return fail(c, AVL_ECUDA, "internal check of the marker layout failed");
    return AVL_OK;
}

// grids and tables of a 1d3v species (the markers come with plan_layout3):
// f, the two deposit accumulators, |v|^2 per velocity cell, the finalize
// partial sums (FIN3_X columns x rq velocity cells per block) and the shift
// tables the field kernel writes for every species
avl_status create_species3(avl_ctx* c, int s, const avl_species& p, int& fin_base)
{
    StepArgs& h = c->h;
    SpDev& sp = h.sp[s];
    const int nx = c->dom.nx;
    const size_t pb = prec_bytes(h.prec);
    sp.nvdim = 3;
    sp.nx = nx;
    sp.nvflat = 1;
    for (int d = 0; d < 3; ++d) {
        sp.nv[d] = p.nv[d];
        sp.nvflat *= p.nv[d];
        sp.vmin[d] = p.vmin[d];
        sp.dv[d] = (p.vmax[d] - p.vmin[d]) / p.nv[d];
        sp.inv_dv[d] = 1.0 / sp.dv[d];
    }
    sp.mobile = p.mobile ? 1 : 0;
    sp.q = p.q;
    sp.m = p.m;
    sp.qm = p.q / p.m;
    sp.dx = c->dom.L / nx;
    sp.qm_dt = sp.qm * c->dom.dt;
    sp.dt_dx = c->dom.dt / sp.dx;
    sp.nchunk = 0;
    sp.npen = 0;
    sp.n = 0;
    sp.nxb = (nx + FIN3_X - 1) / FIN3_X;
    const int nrq0 = std::max(1, (16 * c->num_sms + c->ns * sp.nxb - 1) / (c->ns * sp.nxb));
    int rq = std::max(1, (sp.nvflat + nrq0 - 1) / nrq0);
    const int rq_env = env_int("AVL_RQ", 0);
    if (rq_env > 0) rq = std::min(rq_env, sp.nvflat);
    sp.rq = rq;
    sp.nrq = (sp.nvflat + rq - 1) / rq;
    sp.nfin = sp.nxb * sp.nrq;
    sp.fin_base = fin_base;
    fin_base += sp.nfin;
    h.nfin_total = fin_base;
    const size_t cells = (size_t)nx * sp.nvflat;
    void *pf, *pa0, *pa1, *pv2, *pr, *pd, *p5, *p6;
    cudaError_t e;
    if ((e = dalloc(c, &pf, cells * pb, true)) || (e = dalloc(c, &pa0, 2 * cells * pb, true)) ||
        (e = dalloc(c, &pa1, 2 * cells * pb, true)) || (e = dalloc(c, &pv2, (size_t)sp.nvflat * pb, false)) ||
        (e = dalloc(c, &pr, (size_t)sp.nrq * nx * 8, true)) || (e = dalloc(c, &pd, (size_t)sp.nfin * 4 * 8, true)) ||
        (e = dalloc(c, &p5, (size_t)nx * 4, true)) || (e = dalloc(c, &p6, (size_t)nx * 4, true)))
        return cuda_fail(c, e, "cudaMalloc(species)");
    sp.fgrid = pf;
    sp.ngrid = nullptr;
    sp.acc[0] = pa0;
    sp.acc[1] = pa1;
    sp.v2row = pv2;
    sp.rho_part = (double*)pr;
    sp.dpart = (double*)pd;
    sp.shift[0] = (int*)p5;
    sp.shift[1] = (int*)p6;
    // |v|^2 at the cell centres, internal order [vz][vy][vx]
    std::vector<double> v2(sp.nvflat);
    for (int kz = 0; kz < sp.nv[2]; ++kz)
        for (int ky = 0; ky < sp.nv[1]; ++ky)
            for (int kx = 0; kx < sp.nv[0]; ++kx) {
                const double vx = sp.vmin[0] + (kx + 0.5) * sp.dv[0];
                const double vy = sp.vmin[1] + (ky + 0.5) * sp.dv[1];
                const double vz = sp.vmin[2] + (kz + 0.5) * sp.dv[2];
                v2[((size_t)kz * sp.nv[1] + ky) * sp.nv[0] + kx] = vx * vx + vy * vy + vz * vz;
            }
    if (h.prec == AVL_FP32) {
        std::vector<float> v2f(v2.begin(), v2.end());
        AVL_CUDA(c, cudaMemcpyAsync(pv2, v2f.data(), v2f.size() * 4, cudaMemcpyHostToDevice, c->st));
        AVL_CUDA(c, cudaStreamSynchronize(c->st));
    } else {
        AVL_CUDA(c, cudaMemcpyAsync(pv2, v2.data(), v2.size() * 8, cudaMemcpyHostToDevice, c->st));
        AVL_CUDA(c, cudaStreamSynchronize(c->st));
    }
    return AVL_OK;
}

// the batch's device map (run arguments, block prefixes) and kernel limits,
// rebuilt when a run's launch shapes changed; invalidates the step graph
avl_status ensure_batch_map(avl_ctx* b)
{
    const int nrun = (int)b->runs.size();
    bool ok = b->bm_mem != nullptr && (int)b->bm_versions.size() == nrun;
    for (int r = 0; ok && r < nrun; ++r) ok = b->bm_versions[r] == b->runs[r]->layout_version;
    if (ok) return AVL_OK;
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    AVL_CUDA(b, cudaStreamSynchronize(b->st));
    if (b->bm_mem) {
        cudaFree(b->bm_mem);
        b->bm_mem = nullptr;
    }
    // layout: BatchMap | args[nrun] | pd_base[nrun + 1] | fin_base[nrun + 1]
    const size_t off_args = (sizeof(BatchMap) + 15) / 16 * 16;
    const size_t off_pd = off_args + (size_t)nrun * sizeof(void*);
    const size_t off_fin = off_pd + (size_t)(nrun + 1) * 4;
    const size_t bytes = off_fin + (size_t)(nrun + 1) * 4;
    std::vector<unsigned char> hostbuf(bytes, 0);
    AVL_CUDA(b, cudaMalloc(&b->bm_mem, bytes));
    unsigned char* dbase = static_cast<unsigned char*>(b->bm_mem);
    BatchMap bm;
    bm.nrun = nrun;
    bm.args = reinterpret_cast<const StepArgs* const*>(dbase + off_args);
    bm.pd_base = reinterpret_cast<const int*>(dbase + off_pd);
    bm.fin_base = reinterpret_cast<const int*>(dbase + off_fin);
    memcpy(hostbuf.data(), &bm, sizeof(bm));
    const StepArgs** args = reinterpret_cast<const StepArgs**>(hostbuf.data() + off_args);
    int* pd = reinterpret_cast<int*>(hostbuf.data() + off_pd);
    int* fin = reinterpret_cast<int*>(hostbuf.data() + off_fin);
    pd[0] = fin[0] = 0;
    int pd_smem = 1024, field_smem = 0;
    b->bm_versions.assign(nrun, 0);
    for (int r = 0; r < nrun; ++r) {
        const avl_ctx* c = b->runs[r];
        args[r] = c->d_args;
        pd[r + 1] = pd[r] + c->h.nchunk_total;
        fin[r + 1] = fin[r] + c->h.nfin_total;
        pd_smem = std::max(pd_smem, pd1_smem_needed(c->h));
        field_smem = std::max(field_smem, (int)field_smem_bytes(c->h));
        b->bm_versions[r] = c->layout_version;
    }
    AVL_CUDA(b, cudaMemcpyAsync(b->bm_mem, hostbuf.data(), bytes, cudaMemcpyHostToDevice, b->st));
    AVL_CUDA(b, cudaStreamSynchronize(b->st));
    b->bm_pd_blocks = pd[nrun];
    b->bm_fin_blocks = fin[nrun];
    b->bm_pd_smem = pd_smem;
    b->bm_field_smem = field_smem;
    AVL_CUDA(b, configure_batch1(b->h.prec, pd_smem, field_smem));
    return AVL_OK;
}

// one step of every run: re-sort (where marked), push + deposit, finalize,
// field (one launch each)
avl_status enqueue_batch_step(avl_ctx* b)
{
    const BatchMap* bm = static_cast<const BatchMap*>(b->bm_mem);
    AVL_CUDA(b, launch_rs1_batch(b->h.prec, bm, b->bm_pd_blocks, b->st));
    AVL_CUDA(b, launch_pd1_batch(b->h.prec, bm, b->bm_pd_blocks, b->bm_pd_smem, 1, b->st));
    AVL_CUDA(b, launch_fin1_batch(b->h.prec, bm, b->bm_fin_blocks, 0, b->st));
    AVL_CUDA(b, launch_field_batch(bm, (int)b->runs.size(), b->bm_field_smem, 1, b->st));
    return AVL_OK;
}

}  // namespace

// error reporting for the context-free entry points of other translation units
avl_status avl_noalloc_fail(avl_status st, const char* msg) { return fail(nullptr, st, msg); }

extern "C" {

const char* avl_last_error(const avl_ctx* ctx)
{
    return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

avl_status avl_create(const avl_domain* dom, const avl_species* spec, int32_t nspecies, void* cuda_stream,
                      avl_ctx** out)
{
    if (!out) return fail(nullptr, AVL_EINVAL, "out is NULL");
    *out = nullptr;
    if (!dom || !spec) return fail(nullptr, AVL_EINVAL, "dom or species is NULL");
    if (dom->nvdim != 1 && dom->nvdim != 3) return fail(nullptr, AVL_EINVAL, "nvdim must be 1 or 3");
    if (dom->nx < 4 || dom->nx > (1 << 20)) return fail(nullptr, AVL_EINVAL, "nx must be in [4, 2^20]");
    if (dom->nvdim == 3 && (dom->precision == AVL_FP32 || dom->precision == AVL_FP64) &&
        (dom->nx > (dom->precision == AVL_FP32 ? 1024 : 512) ||
         pd3_smem_bytes(dom->nx, NV3_MAX + 1, dom->precision) > 220 * 1024))
        return fail(nullptr, AVL_EINVAL, "1d3v needs nx <= 1024 (FP32) or nx <= 512 (FP64)");
    if (!(dom->L > 0) || !(dom->dt > 0) || !(dom->poisson_const > 0) || !isfinite(dom->L) ||
        !isfinite(dom->dt) || !isfinite(dom->poisson_const))
        return fail(nullptr, AVL_EINVAL, "L, dt and poisson_const must be positive and finite");
    if (dom->softening != 0 && dom->softening != 1) return fail(nullptr, AVL_EINVAL, "softening must be 0 or 1");
    if (dom->precision != AVL_FP64 && dom->precision != AVL_FP32)
        return fail(nullptr, AVL_EINVAL, "precision must be AVL_FP64 or AVL_FP32");
    if (nspecies < 1 || nspecies > MAXS) return fail(nullptr, AVL_EINVAL, "nspecies must be in [1, 8]");
    for (int s = 0; s < nspecies; ++s) {
        const avl_species& p = spec[s];
        if (!(p.m > 0) || !isfinite(p.q) || !isfinite(p.m))
            return fail(nullptr, AVL_EINVAL, "species mass must be positive, charge finite");
        if (dom->nvdim == 1) {
            if (p.nv[0] < 2 || p.nv[0] > (1 << 20) || p.nv[1] != 1 || p.nv[2] != 1)
                return fail(nullptr, AVL_EINVAL, "1d1v species need nv[0] in [2, 2^20] and nv[1] = nv[2] = 1");
        } else {
            if (p.nv[0] < 2 || p.nv[0] > NV3_MAX || p.nv[1] < 2 || p.nv[1] > 4096 || p.nv[2] < 2 ||
                p.nv[2] > 4096)
                return fail(nullptr, AVL_EINVAL, "1d3v species need nv[0] in [2, 1024], nv[1], nv[2] in [2, 4096]");
            const long long cells = (long long)dom->nx * p.nv[0] * p.nv[1] * p.nv[2];
            if (cells >= (1ll << 31)) return fail(nullptr, AVL_EINVAL, "1d3v grid must have fewer than 2^31 cells");
        }
        for (int d = 0; d < dom->nvdim; ++d)
            if (!(p.vmax[d] > p.vmin[d]) || !isfinite(p.vmin[d]) || !isfinite(p.vmax[d]))
                return fail(nullptr, AVL_EINVAL, "species velocity range must satisfy vmin < vmax");
    }

    avl_ctx* c = new avl_ctx();
    c->dom = *dom;
    c->ns = nspecies;
    for (int s = 0; s < nspecies; ++s) c->sp[s] = spec[s];
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(nullptr, e, "cudaGetDevice");
    }
    if (cuda_stream) {
        c->st = static_cast<cudaStream_t>(cuda_stream);
    } else {
        e = cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            return cuda_fail(nullptr, e, "cudaStreamCreate");
        }
        c->own_stream = true;
    }

    auto bail = [&](avl_status st) {
        std::string m = c->err;
        avl_destroy(c);
        return fail(nullptr, st, m);
    };

    StepArgs& h = c->h;
    memset(&h, 0, sizeof(h));
    h.ns = nspecies;
    h.prec = dom->precision;
    h.nvdim = dom->nvdim;
    const int nx = dom->nx;
    const double dx = dom->L / nx;
    const size_t pb = prec_bytes(h.prec);

    // --- field arrays and spectral multipliers ---------------------------
    FieldDev& fd = h.fd;
    fd.nx = nx;
    fd.pow2 = (nx >= 4 && (nx & (nx - 1)) == 0) ? 1 : 0;
    fd.softening = dom->softening;
    fd.ndiag = 3 + 3 * nspecies;
    fd.resort_drift = env_int("AVL_RESORT_DRIFT", 0) != 0 ? 1 : 0;
    fd.resort_miss = std::max(1, env_int("AVL_RESORT_MISS", 30));
    fd.L = dom->L;
    fd.dx = dx;
    fd.cP = dom->poisson_const;
    fd.we_scale = dx / (2.0 * dom->poisson_const);
    std::vector<double2> tw(nx);
    std::vector<double> gm(nx / 2 + 1, 0.0);
    spectral_tables(nx, dom->L, dom->poisson_const, dom->softening, tw.data(), gm.data());
    void *p_rho, *p_E64, *p_E32, *p_tw, *p_gm, *p_diag;
    if ((e = dalloc(c, &p_rho, nx * 8, true)) || (e = dalloc(c, &p_E64, nx * 8, true)) ||
        (e = dalloc(c, &p_E32, nx * 4, true)) || (e = dalloc(c, &p_tw, nx * 16, false)) ||
        (e = dalloc(c, &p_gm, (nx / 2 + 1) * 8, false)) || (e = dalloc(c, &p_diag, fd.ndiag * 8, true))) {
        cuda_fail(c, e, "cudaMalloc(field)");
        return bail(AVL_ENOMEM);
    }
    fd.green = nullptr;
    if (nx <= GREEN_MAX) {
        std::vector<double> G(nx);
        green_table(nx, gm.data(), G.data());
        void* p_g = nullptr;
        if ((e = dalloc(c, &p_g, nx * 8, false)) ||
            (e = cudaMemcpyAsync(p_g, G.data(), nx * 8, cudaMemcpyHostToDevice, c->st)) ||
            (e = cudaStreamSynchronize(c->st))) {
            cuda_fail(c, e, "Green's function table");
            return bail(AVL_ECUDA);
        }
        fd.green = (const double*)p_g;
    }
    fd.rho = (double*)p_rho;
    fd.E64 = (double*)p_E64;
    fd.E32 = (float*)p_E32;
    fd.tw = (const double2*)p_tw;
    fd.gmul = (const double*)p_gm;
    fd.diag = (double*)p_diag;
    if ((e = cudaMemcpyAsync(p_tw, tw.data(), nx * 16, cudaMemcpyHostToDevice, c->st)) ||
        (e = cudaMemcpyAsync(p_gm, gm.data(), (nx / 2 + 1) * 8, cudaMemcpyHostToDevice, c->st)) ||
        (e = cudaStreamSynchronize(c->st))) {
        cuda_fail(c, e, "upload spectral tables");
        return bail(AVL_ECUDA);
    }

    // --- per species grids and tables ------------------------------------
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) == cudaSuccess && sms > 0)
        c->num_sms = sms;
    int fin_base = 0;
    for (int s = 0; s < nspecies && dom->nvdim == 3; ++s) {
        avl_status st3 = create_species3(c, s, spec[s], fin_base);
        if (st3 != AVL_OK) return bail(st3);
    }
    for (int s = 0; s < nspecies && dom->nvdim == 1; ++s) {
        const avl_species& p = spec[s];
        SpDev& sp = h.sp[s];
        sp.nvdim = 1;
        sp.nx = nx;
        sp.nv[0] = p.nv[0];
        sp.nv[1] = sp.nv[2] = 1;
        sp.nvflat = p.nv[0];
        sp.mobile = p.mobile ? 1 : 0;
        sp.q = p.q;
        sp.m = p.m;
        sp.qm = p.q / p.m;
        sp.dx = dx;
        for (int d = 0; d < 3; ++d) {
            sp.vmin[d] = d == 0 ? p.vmin[0] : -0.5;
            sp.dv[d] = d == 0 ? (p.vmax[0] - p.vmin[0]) / p.nv[0] : 1.0;
            sp.inv_dv[d] = 1.0 / sp.dv[d];
        }
        sp.qm_dt = sp.qm * dom->dt;
        sp.dt_dx = dom->dt / dx;
        sp.nchunk = 0;
        sp.n = 0;
        // finalize blocks: FIN_XB columns x rq rows, about 4 blocks per SM in total
        sp.nxb = (nx + FIN_XB - 1) / FIN_XB;
        const int nrq = std::max(1, (4 * c->num_sms + nspecies * sp.nxb - 1) / (nspecies * sp.nxb));
        int rq = std::max(8, (p.nv[0] + nrq - 1) / nrq);
        const int rq_env = env_int("AVL_RQ", 0);
        if (rq_env > 0) rq = rq_env;
        rq = std::min(rq, p.nv[0]);
        sp.rq = rq;
        sp.nrq = (p.nv[0] + rq - 1) / rq;
        sp.nfin = sp.nxb * sp.nrq;
        sp.fin_base = fin_base;
        fin_base += sp.nfin;
        const size_t cells = (size_t)nx * sp.nvflat;
        const size_t nvk = (size_t)sp.nvflat;
        void *pf, *pn, *po, *pr, *pd, *p1, *p2, *p3, *p4, *p5, *p6;
        if ((e = dalloc(c, &pf, cells * pb, true)) || (e = dalloc(c, &pn, cells * pb, true)) ||
            (e = dalloc(c, &po, 2 * cells * 8 + nvk * 8, true)) || (e = dalloc(c, &pr, (size_t)sp.nrq * nx * 8, true)) ||
            (e = dalloc(c, &pd, (size_t)sp.nfin * 4 * 8, true)) || (e = dalloc(c, &p1, nvk * 4, true)) ||
            (e = dalloc(c, &p2, nvk * 4, true)) || (e = dalloc(c, &p3, (nvk + 1) * 4, true)) ||
            (e = dalloc(c, &p4, nvk * 4, true)) || (e = dalloc(c, &p5, (size_t)nx * 4, true)) ||
            (e = dalloc(c, &p6, (size_t)nx * 4, true))) {
            cuda_fail(c, e, "cudaMalloc(species)");
            return bail(AVL_ENOMEM);
        }
        sp.fgrid = pf;
        sp.ngrid = pn;
        sp.ovf = (double*)po;
        sp.ovf_tag = reinterpret_cast<int*>(sp.ovf + 2 * cells);
        sp.rho_part = (double*)pr;
        sp.dpart = (double*)pd;
        sp.far_cnt[0] = (int*)p1;
        sp.far_cnt[1] = (int*)p4;
        sp.far_cur = (int*)p2;
        sp.base_new = (int*)p3;
        sp.shift[0] = (int*)p5;
        sp.shift[1] = (int*)p6;
    }
    h.nchunk_total = 0;
    h.nfin_total = fin_base;

    void *pa, *pc, *pf0, *pbad, *plog;
    if ((e = dalloc(c, &pa, sizeof(StepArgs), false)) || (e = dalloc(c, &pc, sizeof(Ctl), true)) ||
        (e = dalloc(c, &pf0, sizeof(avl_f0), false)) || (e = dalloc(c, &pbad, 8, true)) ||
        (e = dalloc(c, &plog, LOG_TAB_N * sizeof(double2), false))) {
        cuda_fail(c, e, "cudaMalloc(control)");
        return bail(AVL_ENOMEM);
    }
    h.fd.logtab = (const double2*)plog;
    if ((e = init_log_table((double2*)plog, c->st))) {
        cuda_fail(c, e, "avl_create (logarithm table)");
        return bail(AVL_ECUDA);
    }
    c->d_args = (StepArgs*)pa;
    c->d_ctl = (Ctl*)pc;
    c->d_f0 = (avl_f0*)pf0;
    c->d_bad = (unsigned long long*)pbad;
    h.ctl = c->d_ctl;
    {
        const long long wl = WAIT_LIMIT;
        if ((e = cudaMemcpyAsync(&c->d_ctl->wait_limit, &wl, sizeof(wl), cudaMemcpyHostToDevice, c->st)) ||
            (e = cudaStreamSynchronize(c->st))) {
            cuda_fail(c, e, "avl_create (control block)");
            return bail(AVL_ECUDA);
        }
    }
    // only the deposit kernels of the context's velocity dimension (the other
    // dimension's shared memory at this nx may exceed what a CTA can hold)
    if ((e = dom->nvdim == 1 ? configure_vhs1(h) : configure_vhs3(h)) || (e = configure_field(h))) {
        cuda_fail(c, e, "cudaFuncSetAttribute (shared memory)");
        return bail(AVL_ECUDA);
    }
    if (upload_args(c) != AVL_OK) return bail(AVL_ECUDA);
    *out = c;
    return AVL_OK;
}

void avl_destroy(avl_ctx* c)
{
    if (!c || c->parent) return;   // a run belongs to its batch
    for (avl_ctx* r : c->runs) {
        r->parent = nullptr;
        avl_destroy(r);
    }
    if (c->bm_mem) {
        if (c->st) cudaStreamSynchronize(c->st);
        cudaFree(c->bm_mem);
    }
    if (c->st) cudaStreamSynchronize(c->st);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    adjoint_free(c->adj);
    for (void* p : c->allocs) cudaFree(p);
    for (int s = 0; s < MAXS; ++s) free_layout(c, s);
    if (c->scratch) cudaFree(c->scratch);
    if (c->hist_mem) cudaFree(c->hist_mem);
    if (c->own_stream && c->st) cudaStreamDestroy(c->st);
    delete c;
}

avl_status avl_init_markers(avl_ctx* c, int32_t s, const int32_t lattice[4], const avl_f0* f0, uint64_t seed,
                            double jitter)
{
    avl_status st = check_species(c, s);
    if (st) return st;
    if (!lattice || !f0) return fail(c, AVL_EINVAL, "lattice or f0 is NULL");
    const int nvd = c->h.nvdim;
    if (nvd == 1 && (lattice[0] < 1 || lattice[1] < 1 || lattice[2] != 1 || lattice[3] != 1))
        return fail(c, AVL_EINVAL, "1d1v lattice must be {px >= 1, pv >= 1, 1, 1}");
    if (nvd == 3 && (lattice[0] < 1 || lattice[1] < 1 || lattice[2] < 1 || lattice[3] < 1 ||
                     (long long)lattice[0] * lattice[1] * lattice[2] * lattice[3] > 4096))
        return fail(c, AVL_EINVAL, "1d3v lattice must be {px, pvx, pvy, pvz} >= 1 with at most 4096 points");
    if (f0->nbeam < 1 || f0->nbeam > 4 || f0->nmode < 0 || f0->nmode > 64)
        return fail(c, AVL_EINVAL, "f0 needs 1..4 beams and 0..64 modes");
    for (int b = 0; b < f0->nbeam; ++b)
        for (int d = 0; d < nvd; ++d)
            if (!(f0->beam_vth[b][d] > 0)) return fail(c, AVL_EINVAL, "beam thermal speeds must be positive");
    if (!(jitter >= 0.0 && jitter <= 1.0)) return fail(c, AVL_EINVAL, "jitter must be in [0, 1]");
    SpDev& sp = c->h.sp[s];
    const long long ppc = (long long)lattice[0] * lattice[1] * lattice[2] * lattice[3];
    const long long n = (long long)sp.nx * sp.nvflat * ppc;
    if (n >= (1ll << 31) - 1024) return fail(c, AVL_EINVAL, "too many markers for one species (2^31)");
    if ((st = nvd == 3 ? plan_layout3(c, s, n) : plan_layout(c, s, n))) return st;
    if ((st = set_cur_zero(c, s))) return st;
    AVL_CUDA(c, cudaMemcpyAsync(c->d_f0, f0, sizeof(avl_f0), cudaMemcpyHostToDevice, c->st));
    if ((st = upload_args(c))) return st;
    if (nvd == 3)
        AVL_CUDA(c, launch_init3(c->h, c->d_args, s, lattice, c->d_f0, seed, jitter, c->st));
    else
        AVL_CUDA(c, launch_init1(c->h, c->d_args, s, lattice, c->d_f0, seed, jitter, c->st));
    c->has_markers[s] = true;
    c->lattice_made[s] = true;
    c->refinable[s] = true;
    {
        long long step = 0;
        AVL_CUDA(c, cudaMemcpyAsync(&step, &c->d_ctl->step, 8, cudaMemcpyDeviceToHost, c->st));
        AVL_CUDA(c, cudaStreamSynchronize(c->st));
        c->init_step[s] = step;
    }
    for (int d = 0; d < 4; ++d) c->lat[s][d] = lattice[d];
    c->seed_s[s] = seed;
    c->jitter_s[s] = jitter;
    c->f0_s[s] = *f0;
    if ((st = refresh(c))) return st;
    return read_errors(c);
}

avl_status avl_set_markers(avl_ctx* c, int32_t s, int64_t n, const double* x, const double* v, const double* f,
                           int32_t on_device)
{
    avl_status st = check_species(c, s);
    if (st) return st;
    if (n <= 0 || n >= (1ll << 31) - 1024) return fail(c, AVL_EINVAL, "n must be in [1, 2^31)");
    if (!x || !v || !f) return fail(c, AVL_EINVAL, "x, v or f is NULL");
    const double *dx_ = x, *dv_ = v, *df_ = f;
    const int nvd = c->h.nvdim;
    if (!on_device) {
        if ((st = ensure_scratch(c, (size_t)n * 8 * (2 + nvd)))) return st;
        double* base = static_cast<double*>(c->scratch);
        AVL_CUDA(c, cudaMemcpyAsync(base, x, n * 8, cudaMemcpyHostToDevice, c->st));
        AVL_CUDA(c, cudaMemcpyAsync(base + n, v, n * 8 * nvd, cudaMemcpyHostToDevice, c->st));
        AVL_CUDA(c, cudaMemcpyAsync(base + n * (1 + nvd), f, n * 8, cudaMemcpyHostToDevice, c->st));
        dx_ = base;
        dv_ = base + n;
        df_ = base + n * (1 + nvd);
    }
    c->lattice_made[s] = false;
    c->refinable[s] = false;
    if ((st = nvd == 3 ? plan_layout3(c, s, n) : plan_layout(c, s, n))) return st;
    if ((st = set_cur_zero(c, s))) return st;
    if ((st = upload_args(c))) return st;
    AVL_CUDA(c, cudaMemsetAsync(c->d_bad, 0, 8, c->st));
    if (nvd == 3)
        AVL_CUDA(c, launch_set3(c->h, c->d_args, s, n, dx_, dv_, df_, c->d_bad, c->st));
    else
        AVL_CUDA(c, launch_set1(c->h, c->d_args, s, n, dx_, dv_, df_, c->d_bad, c->st));
    unsigned long long bad = 0;
    AVL_CUDA(c, cudaMemcpyAsync(&bad, c->d_bad, 8, cudaMemcpyDeviceToHost, c->st));
    AVL_CUDA(c, cudaStreamSynchronize(c->st));
    if (bad) {
        c->has_markers[s] = false;
        return fail(c, AVL_EINVAL, "markers with x outside [0, L) or non-finite values: " + std::to_string(bad));
    }
    c->has_markers[s] = true;
    if ((st = refresh(c))) return st;
    return read_errors(c);
}

avl_status avl_marker_count(avl_ctx* c, int32_t s, int64_t* n)
{
    avl_status st = check_species(c, s);
    if (st) return st;
    if (!n) return fail(c, AVL_EINVAL, "n is NULL");
    *n = c->has_markers[s] ? c->h.sp[s].n : 0;
    return AVL_OK;
}

avl_status avl_get_markers(avl_ctx* c, int32_t s, double* x, double* v, double* f, int32_t on_device)
{
    avl_status st = check_species(c, s);
    if (st) return st;
    if (!c->has_markers[s]) return fail(c, AVL_ESTATE, "species has no markers");
    const long long n = c->h.sp[s].n;
    const int nvd = c->h.nvdim;
    auto get = [&](double* gx, double* gv, double* gf) {
        return nvd == 3 ? launch_get3(c->h, c->d_args, s, gx, gv, gf, c->st)
                        : launch_get1(c->h, c->d_args, s, gx, gv, gf, c->st);
    };
    if (on_device) {
        AVL_CUDA(c, get(x, v, f));
        return AVL_OK;
    }
    if ((st = ensure_scratch(c, (size_t)n * 8 * (2 + nvd)))) return st;
    double* base = static_cast<double*>(c->scratch);
    AVL_CUDA(c, get(base, base + n, base + n * (1 + nvd)));
    if (x) AVL_CUDA(c, cudaMemcpyAsync(x, base, n * 8, cudaMemcpyDeviceToHost, c->st));
    if (v) AVL_CUDA(c, cudaMemcpyAsync(v, base + n, n * 8 * nvd, cudaMemcpyDeviceToHost, c->st));
    if (f) AVL_CUDA(c, cudaMemcpyAsync(f, base + n * (1 + nvd), n * 8, cudaMemcpyDeviceToHost, c->st));
    AVL_CUDA(c, cudaStreamSynchronize(c->st));
    return AVL_OK;
}

avl_status avl_step(avl_ctx* c, int32_t nsteps)
{
    if (!c) return AVL_EINVAL;
    if (nsteps < 0) return fail(c, AVL_EINVAL, "nsteps must be >= 0");
    for (int s = 0; s < c->ns; ++s)
        if (c->h.sp[s].mobile && !c->has_markers[s])
            return fail(c, AVL_ESTATE, "mobile species " + std::to_string(s) + " has no markers");
    for (size_t r = 0; r < c->runs.size(); ++r)
        for (int s = 0; s < c->runs[r]->ns; ++s)
            if (c->runs[r]->h.sp[s].mobile && !c->runs[r]->has_markers[s])
                return fail(c, AVL_ESTATE, "run " + std::to_string(r) + ": mobile species " + std::to_string(s) +
                                               " has no markers");
    if (nsteps == 0) return AVL_OK;
    if (!c->runs.empty()) {
        avl_status st = ensure_batch_map(c);
        if (st) return st;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    AVL_CUDA(c, cudaStreamIsCapturing(c->st, &cap));
    if (cap != cudaStreamCaptureStatusNone || env_int("AVL_NO_GRAPH", 0)) {
        for (int i = 0; i < nsteps; ++i) {
            avl_status st = enqueue_step(c);
            if (st) return st;
        }
        return AVL_OK;
    }
    avl_status st = build_graph(c);
    if (st) return st;
    for (int i = 0; i < nsteps; ++i) AVL_CUDA(c, cudaGraphLaunch(c->gexec, c->st));
    return AVL_OK;
}

avl_status avl_record_history(avl_ctx* c, int32_t max_steps)
{
    if (!c) return AVL_EINVAL;
    if (!c->runs.empty()) return fail(c, AVL_EINVAL, "record the history on the runs of a batch, not the batch");
    if (max_steps < 1 || max_steps > (1 << 24)) return fail(c, AVL_EINVAL, "max_steps must be in [1, 2^24]");
    const int nx = c->h.fd.nx;
    AVL_CUDA(c, cudaStreamSynchronize(c->st));
    if (c->hist_mem) {
        cudaFree(c->hist_mem);
        c->hist_mem = nullptr;
        c->h.fd.hist = nullptr;
    }
    const size_t bytes = ((size_t)max_steps + 1) * nx * 8;
    cudaError_t e = cudaMalloc(&c->hist_mem, bytes);
    if (e) {
        c->hist_mem = nullptr;
        upload_args(c);
        return cuda_fail(c, e, "cudaMalloc(field history)");
    }
    long long step = 0;
    AVL_CUDA(c, cudaMemcpyAsync(&step, &c->d_ctl->step, 8, cudaMemcpyDeviceToHost, c->st));
    AVL_CUDA(c, cudaMemcpyAsync(c->hist_mem, c->h.fd.E64, (size_t)nx * 8, cudaMemcpyDeviceToDevice, c->st));
    AVL_CUDA(c, cudaStreamSynchronize(c->st));
    c->h.fd.hist = static_cast<double*>(c->hist_mem);
    c->h.fd.hist_cap = max_steps + 1;
    c->h.fd.hist_origin = step;
    return upload_args(c);
}

avl_status avl_refine_markers(avl_ctx* c, int32_t s, const int32_t* box, const int32_t* lattice, uint64_t seed,
                              double jitter, int64_t* added)
{
    avl_status st = check_species(c, s);
    if (st) return st;
    if (added) *added = 0;
    if (!box || !lattice) return fail(c, AVL_EINVAL, "box or lattice is NULL");
    if (c->h.nvdim != 1) return fail(c, AVL_EINVAL, "marker refinement is 1d1v");
    const SpDev& sp = c->h.sp[s];
    if (!(box[0] >= 0 && box[0] < box[1] && box[1] <= sp.nx && box[2] >= 0 && box[2] < box[3] &&
          box[3] <= sp.nvflat))
        return fail(c, AVL_EINVAL, "box must satisfy 0 <= x0 < x1 <= nx and 0 <= v0 < v1 <= nv");
    if (lattice[0] < 1 || lattice[1] < 1 || (long long)lattice[0] * lattice[1] > 4096)
        return fail(c, AVL_EINVAL, "lattice must be {px, pv} >= 1 with at most 4096 points");
    if (!(jitter >= 0.0 && jitter <= 1.0)) return fail(c, AVL_EINVAL, "jitter must be in [0, 1]");
    if (!c->refinable[s])
        return fail(c, AVL_ESTATE, "species markers were not created by avl_init_markers (no initial f0 to trace to)");
    const FieldDev& fd = c->h.fd;
    if (!fd.hist) return fail(c, AVL_ESTATE, "no field history: call avl_record_history before avl_init_markers");
    long long step = 0;
    AVL_CUDA(c, cudaMemcpyAsync(&step, &c->d_ctl->step, 8, cudaMemcpyDeviceToHost, c->st));
    AVL_CUDA(c, cudaStreamSynchronize(c->st));
    const long long first = c->init_step[s] - fd.hist_origin, nhist = step - c->init_step[s];
    if (first < 0 || first + nhist > fd.hist_cap)
        return fail(c, AVL_ESTATE, "the field history does not cover every step since the species' markers were created");
    const long long count = (long long)(box[1] - box[0]) * (box[3] - box[2]) * lattice[0] * lattice[1];
    const long long n_old = sp.n, n_new = n_old + count;
    if (n_new >= (1ll << 31) - 1024) return fail(c, AVL_EINVAL, "too many markers for one species (2^31)");
    if ((st = ensure_scratch(c, (size_t)n_new * 24))) return st;
    double* x = static_cast<double*>(c->scratch);
    double* v = x + n_new;
    double* f = v + n_new;
    AVL_CUDA(c, launch_get1(c->h, c->d_args, s, x, v, f, c->st));
    AVL_CUDA(c, cudaMemcpyAsync(c->d_f0, &c->f0_s[s], sizeof(avl_f0), cudaMemcpyHostToDevice, c->st));
    const int b[4] = {box[0], box[1], box[2], box[3]}, lat[2] = {lattice[0], lattice[1]};
    AVL_CUDA(c, launch_refine1(c->h, s, b, lat, c->d_f0, seed, jitter, c->dom.dt, (int)nhist,
                               fd.hist + first * fd.nx, count, x + n_old, v + n_old, f + n_old, c->st));
    // the whole set into a fresh layout (re-sorted, reconstructed, field solved)
    // (avl_set_markers clears the creation lattice: the adjoint needs its order)
    const long long init_step = c->init_step[s];
    if ((st = avl_set_markers(c, s, n_new, x, v, f, 1))) return st;
    c->refinable[s] = true;
    c->init_step[s] = init_step;
    if (added) *added = count;
    return AVL_OK;
}

avl_status avl_set_bfield(avl_ctx* c, const double* B)
{
    if (!c) return AVL_EINVAL;
    if (c->h.nvdim != 3) return fail(c, AVL_EINVAL, "a magnetic field needs nvdim = 3");
    if (!B) return fail(c, AVL_EINVAL, "B is NULL");
    for (int d = 0; d < 3; ++d)
        if (!isfinite(B[d])) return fail(c, AVL_EINVAL, "B must be finite");
    AVL_CUDA(c, cudaStreamSynchronize(c->st));
    FieldDev& fd = c->h.fd;
    for (int d = 0; d < 3; ++d) fd.B[d] = B[d];
    fd.magnetized = (B[0] != 0.0 || B[1] != 0.0 || B[2] != 0.0) ? 1 : 0;
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return upload_args(c);
}

avl_status avl_get_f(avl_ctx* c, int32_t s, double* f, double* n_opt, int32_t on_device)
{
    avl_status st = check_species(c, s);
    if (st) return st;
    if (!f) return fail(c, AVL_EINVAL, "f is NULL");
    const SpDev& sp = c->h.sp[s];
    const size_t cells = (size_t)sp.nx * sp.nvflat;
    int which = 0;   // 1d3v: accumulator of the last deposit
    if (sp.nvdim == 3) {
        int asel = 0;
        AVL_CUDA(c, cudaMemcpyAsync(&asel, &c->d_ctl->asel[s], sizeof(int), cudaMemcpyDeviceToHost, c->st));
        AVL_CUDA(c, cudaStreamSynchronize(c->st));
        which = 1 - asel;
    }
    auto getf = [&](double* gf, double* gn) {
        return sp.nvdim == 3 ? launch_getf3(c->h, s, which, gf, gn, c->st) : launch_getf(c->h, s, gf, gn, c->st);
    };
    if (on_device) {
        AVL_CUDA(c, getf(f, n_opt));
        return AVL_OK;
    }
    if ((st = ensure_scratch(c, cells * 16))) return st;
    double* base = static_cast<double*>(c->scratch);
    AVL_CUDA(c, getf(base, n_opt ? base + cells : nullptr));
    AVL_CUDA(c, cudaMemcpyAsync(f, base, cells * 8, cudaMemcpyDeviceToHost, c->st));
    if (n_opt) AVL_CUDA(c, cudaMemcpyAsync(n_opt, base + cells, cells * 8, cudaMemcpyDeviceToHost, c->st));
    AVL_CUDA(c, cudaStreamSynchronize(c->st));
    return AVL_OK;
}

static avl_status get_field(avl_ctx* c, const double* src, double* dst, int on_device)
{
    if (!c) return AVL_EINVAL;
    if (!c->runs.empty()) return fail(c, AVL_EINVAL, "a batch has no field; use a run");
    if (!dst) return fail(c, AVL_EINVAL, "output is NULL");
    const size_t bytes = (size_t)c->h.fd.nx * 8;
    AVL_CUDA(c, cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                c->st));
    if (!on_device) AVL_CUDA(c, cudaStreamSynchronize(c->st));
    return AVL_OK;
}

avl_status avl_get_rho(avl_ctx* c, double* rho, int32_t on_device)
{
    return get_field(c, c ? c->h.fd.rho : nullptr, rho, on_device);
}

avl_status avl_get_E(avl_ctx* c, double* E, int32_t on_device)
{
    return get_field(c, c ? c->h.fd.E64 : nullptr, E, on_device);
}

avl_status avl_get_moments(avl_ctx* c, int32_t s, double* out, int32_t on_device)
{
    avl_status st = check_species(c, s);
    if (st) return st;
    if (!out) return fail(c, AVL_EINVAL, "out is NULL");
    const SpDev& sp = c->h.sp[s];
    const size_t bytes = (size_t)(2 + sp.nvdim) * sp.nx * 8;
    if (on_device) {
        AVL_CUDA(c, launch_moments(c->h, c->d_args, s, out, c->st));
        return AVL_OK;
    }
    if ((st = ensure_scratch(c, bytes))) return st;
    AVL_CUDA(c, launch_moments(c->h, c->d_args, s, static_cast<double*>(c->scratch), c->st));
    AVL_CUDA(c, cudaMemcpyAsync(out, c->scratch, bytes, cudaMemcpyDeviceToHost, c->st));
    AVL_CUDA(c, cudaStreamSynchronize(c->st));
    return AVL_OK;
}

avl_status avl_get_residual(avl_ctx* c, double* out, int32_t on_device)
{
    if (!c || !c->runs.empty()) return c ? fail(c, AVL_EINVAL, "a batch has no field; use a run") : AVL_EINVAL;
    if (!out) return fail(c, AVL_EINVAL, "out is NULL");
    const size_t bytes = (size_t)c->h.fd.nx * 8;
    if (on_device) {
        AVL_CUDA(c, launch_residual(c->h, c->d_args, out, c->st));
        return AVL_OK;
    }
    avl_status st = ensure_scratch(c, bytes);
    if (st) return st;
    AVL_CUDA(c, launch_residual(c->h, c->d_args, static_cast<double*>(c->scratch), c->st));
    AVL_CUDA(c, cudaMemcpyAsync(out, c->scratch, bytes, cudaMemcpyDeviceToHost, c->st));
    AVL_CUDA(c, cudaStreamSynchronize(c->st));
    return AVL_OK;
}

avl_status avl_get_diag(avl_ctx* c, double* out)
{
    if (!c) return AVL_EINVAL;
    if (!c->runs.empty()) return fail(c, AVL_EINVAL, "a batch has no diagnostics row; use a run");
    if (!out) return fail(c, AVL_EINVAL, "out is NULL");
    const int nd = c->h.fd.ndiag;
    AVL_CUDA(c, cudaMemcpyAsync(out, c->h.fd.diag, nd * 8, cudaMemcpyDeviceToHost, c->st));
    AVL_CUDA(c, cudaStreamSynchronize(c->st));
    for (int i = 0; i < nd; ++i)
        if (!isfinite(out[i])) return fail(c, AVL_ENUMERIC, "non-finite diagnostic value");
    return AVL_OK;
}

avl_status avl_get_diag_async(avl_ctx* c, double* out)
{
    if (!c) return AVL_EINVAL;
    if (!c->runs.empty()) return fail(c, AVL_EINVAL, "a batch has no diagnostics row; use a run");
    if (!out) return fail(c, AVL_EINVAL, "out is NULL");
    AVL_CUDA(c, cudaMemcpyAsync(out, c->h.fd.diag, c->h.fd.ndiag * 8, cudaMemcpyDeviceToHost, c->st));
    return AVL_OK;
}

avl_status avl_get_stats(avl_ctx* c, int64_t* out)
{
    if (!c) return AVL_EINVAL;
    if (!out) return fail(c, AVL_EINVAL, "out is NULL");
    Ctl h;
    AVL_CUDA(c, cudaMemcpyAsync(&h, c->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->st));
    AVL_CUDA(c, cudaStreamSynchronize(c->st));
    for (int s = 0; s < c->ns; ++s) {
        out[4 * s + 0] = (int64_t)(c->h.nvdim == 3 ? h.movers_last[s] : h.ovf_last[s]);
        out[4 * s + 1] = (int64_t)h.nsort[s];
        out[4 * s + 2] = (int64_t)h.uncovered[s];
        out[4 * s + 3] = (int64_t)h.step;
    }
    return AVL_OK;
}

avl_status avl_profile_steps(avl_ctx* c, int32_t nsteps, double* ms, int32_t nkernels)
{
    if (!c) return AVL_EINVAL;
    if (!ms || nkernels < 4 || nsteps < 0) return fail(c, AVL_EINVAL, "ms must hold 4 values, nsteps >= 0");
    for (int s = 0; s < c->ns; ++s)
        if (c->h.sp[s].mobile && !c->has_markers[s])
            return fail(c, AVL_ESTATE, "mobile species " + std::to_string(s) + " has no markers");
    const bool batch = !c->runs.empty();
    if (batch) {
        avl_status st0 = ensure_batch_map(c);
        if (st0) return st0;
    }
    const BatchMap* bm = static_cast<const BatchMap*>(c->bm_mem);
    cudaEvent_t ev[5];
    for (int i = 0; i < 5; ++i) AVL_CUDA(c, cudaEventCreate(&ev[i]));
    double acc[4] = {0, 0, 0, 0};
    avl_status st = AVL_OK;
    for (int i = 0; i < nsteps && st == AVL_OK; ++i) {
        const bool d3 = c->h.nvdim == 3, mag = d3 && c->h.fd.magnetized;
        cudaError_t e = cudaEventRecord(ev[0], c->st);
        if (!e)
            e = batch ? launch_rs1_batch(c->h.prec, bm, c->bm_pd_blocks, c->st)
                : d3  ? (mag ? launch_magnetized_push(c) : launch_sort3(c->h, c->d_args, c->st))
                      : launch_rs1(c->h, c->d_args, c->st);
        if (!e) e = cudaEventRecord(ev[1], c->st);
        if (!e)
            e = batch ? launch_pd1_batch(c->h.prec, bm, c->bm_pd_blocks, c->bm_pd_smem, 1, c->st)
                : d3  ? launch_pd3(c->h, c->d_args, mag ? 2 : 1, c->st)
                      : launch_pd1(c->h, c->d_args, 1, c->st);
        if (!e) e = cudaEventRecord(ev[2], c->st);
        if (!e)
            e = batch ? launch_fin1_batch(c->h.prec, bm, c->bm_fin_blocks, 0, c->st)
                : d3  ? launch_fin3(c->h, c->d_args, 0, c->st)
                      : launch_fin1(c->h, c->d_args, 0, c->st);
        if (!e) e = cudaEventRecord(ev[3], c->st);
        if (!e)
            e = batch ? launch_field_batch(bm, (int)c->runs.size(), c->bm_field_smem, 1, c->st)
                      : launch_field(c->h, c->d_args, 1, c->st);
        if (!e) e = cudaEventRecord(ev[4], c->st);
        if (!e) e = cudaEventSynchronize(ev[4]);
        for (int k = 0; k < 4 && !e; ++k) {
            float t = 0.f;
            e = cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
            acc[k] += t;
        }
        if (e) st = cuda_fail(c, e, "avl_profile_steps");
    }
    for (int i = 0; i < 5; ++i) cudaEventDestroy(ev[i]);
    for (int k = 0; k < 4; ++k) ms[k] = acc[k];
    return st;
}

avl_status avl_field_solve(int32_t nx, double L, double poisson_const, int32_t softening, const double* rho,
                           double* E, void* cuda_stream)
{
    if (nx < 4 || nx > (1 << 16)) return fail(nullptr, AVL_EINVAL, "nx must be in [4, 65536]");
    if (!(L > 0) || !(poisson_const > 0) || !isfinite(L) || !isfinite(poisson_const))
        return fail(nullptr, AVL_EINVAL, "L and poisson_const must be positive and finite");
    if (softening != 0 && softening != 1) return fail(nullptr, AVL_EINVAL, "softening must be 0 or 1");
    if (!rho || !E) return fail(nullptr, AVL_EINVAL, "rho or E is NULL");
    if (poisson_smem_bytes(nx) > 200 * 1024) return fail(nullptr, AVL_EINVAL, "nx too large for one block");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    std::vector<double2> tw(nx);
    std::vector<double> gm(nx / 2 + 1);
    spectral_tables(nx, L, poisson_const, softening, tw.data(), gm.data());
    void* tab = nullptr;
    const size_t twb = (size_t)nx * 16, gmb = (size_t)(nx / 2 + 1) * 8;
    cudaError_t e = cudaMalloc(&tab, twb + gmb);
    if (e) return cuda_fail(nullptr, e, "cudaMalloc(spectral tables)");
    double2* dtw = static_cast<double2*>(tab);
    double* dgm = reinterpret_cast<double*>(static_cast<unsigned char*>(tab) + twb);
    e = cudaMemcpyAsync(dtw, tw.data(), twb, cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(dgm, gm.data(), gmb, cudaMemcpyHostToDevice, st);
    if (!e) e = launch_poisson(rho, E, nx, dtw, dgm, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    cudaFree(tab);
    if (e || e2) return cuda_fail(nullptr, e ? e : e2, "avl_field_solve");
    return AVL_OK;
}

avl_status avl_adjoint(avl_ctx* c, int32_t s, const avl_f0* theta, int32_t nsteps, int32_t ckpt_every,
                       double* dJ_damp, double* dJ_ddrift, double* J)
{
    avl_status st = check_species(c, s);
    if (st) return st;
    if (c->h.nvdim != 1) return fail(c, AVL_EINVAL, "avl_adjoint supports 1d1v contexts");
    if (c->h.prec == AVL_FP64 && c->h.fd.nx >= 2048)   // fixed-point positions (PosX)
        return fail(c, AVL_EINVAL, "the FP64 adjoint needs nx < 2048");
    if (!theta || !dJ_damp || !dJ_ddrift || !J) return fail(c, AVL_EINVAL, "theta or an output is NULL");
    if (nsteps < 0 || ckpt_every < 1) return fail(c, AVL_EINVAL, "nsteps must be >= 0 and ckpt_every >= 1");
    if (theta->nbeam < 1 || theta->nbeam > 4 || theta->nmode < 0 || theta->nmode > 64)
        return fail(c, AVL_EINVAL, "theta needs 1..4 beams and 0..64 modes");
    for (int b = 0; b < theta->nbeam; ++b)
        if (!(theta->beam_vth[b][0] > 0)) return fail(c, AVL_EINVAL, "beam thermal speeds must be positive");
    AdjSpec spec{};
    spec.theta_s = s;
    spec.nsteps = nsteps;
    spec.ckpt_every = ckpt_every;
    for (int q = 0; q < c->ns; ++q) {
        if (!c->has_markers[q] || !c->lattice_made[q])
            return fail(c, AVL_ESTATE, "avl_adjoint needs the markers of every species from avl_init_markers");
        spec.n[q] = c->h.sp[q].n;
        spec.lat[q][0] = c->lat[q][0];
        spec.lat[q][1] = c->lat[q][1];
        spec.seed[q] = c->seed_s[q];
        spec.jitter[q] = c->jitter_s[q];
        spec.f0[q] = q == s ? *theta : c->f0_s[q];
    }
    cudaError_t e = adjoint_run(&c->adj, c->h, c->d_args, spec, c->st, dJ_damp, dJ_ddrift, J);
    if (e) return cuda_fail(c, e, "avl_adjoint");
    return read_errors(c);
}

avl_status avl_synchronize(avl_ctx* c)
{
    if (!c) return AVL_EINVAL;
    AVL_CUDA(c, cudaStreamSynchronize(c->st));
    for (size_t r = 0; r < c->runs.size(); ++r) {
        avl_status st = read_errors(c->runs[r]);
        if (st) return fail(c, st, "run " + std::to_string(r) + ": " + c->runs[r]->err);
    }
    return c->runs.empty() ? read_errors(c) : AVL_OK;
}

avl_status avl_create_batch(int32_t nrun, const avl_domain* doms, const avl_species* sps, const int32_t* nspecies,
                            void* cuda_stream, avl_ctx** out)
{
    if (!out) return fail(nullptr, AVL_EINVAL, "out is NULL");
    *out = nullptr;
    if (nrun < 1 || nrun > 4096) return fail(nullptr, AVL_EINVAL, "nrun must be in [1, 4096]");
    if (!doms || !sps || !nspecies) return fail(nullptr, AVL_EINVAL, "doms, sps or nspecies is NULL");
    for (int r = 0; r < nrun; ++r) {
        if (doms[r].nvdim != 1) return fail(nullptr, AVL_EINVAL, "batched runs must be 1d1v");
        if (doms[r].precision != doms[0].precision)
            return fail(nullptr, AVL_EINVAL, "batched runs must share one precision");
    }
    avl_ctx* b = new avl_ctx();
    b->dom = doms[0];
    b->h.prec = doms[0].precision;
    b->h.nvdim = 1;
    cudaError_t e = cudaGetDevice(&b->device);
    if (!e && cuda_stream) {
        b->st = static_cast<cudaStream_t>(cuda_stream);
    } else if (!e) {
        e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking);
        b->own_stream = e == cudaSuccess;
    }
    if (e) {
        delete b;
        return cuda_fail(nullptr, e, "avl_create_batch");
    }
    int off = 0;
    for (int r = 0; r < nrun; ++r) {
        avl_ctx* c = nullptr;
        avl_status st = avl_create(&doms[r], sps + off, nspecies[r], b->st, &c);
        if (st) {
            std::string m = "run " + std::to_string(r) + ": " + g_create_err;
            avl_destroy(b);
            return fail(nullptr, st, m);
        }
        c->parent = b;
        b->runs.push_back(c);
        off += nspecies[r];
    }
    // finalize row groups for the whole launch: each run's were sized as if it
    // filled the GPU alone; about 64 blocks per SM over all runs instead (row
    // groups only grow, so the runs' charge and diagnostics partials still fit)
    if (env_int("AVL_RQ", 0) <= 0) {
        double cells = 0.0;
        for (avl_ctx* c : b->runs)
            for (int s = 0; s < c->ns; ++s) cells += (double)c->h.sp[s].nx * c->h.sp[s].nvflat;
        const double per_block = cells / (64.0 * b->runs[0]->num_sms);
        const int rq_batch = std::max(8, (int)std::ceil(per_block / FIN_XB));
        for (avl_ctx* c : b->runs) {
            int fin_base = 0;
            for (int s = 0; s < c->ns; ++s) {
                SpDev& sp = c->h.sp[s];
                sp.rq = std::min(std::max(sp.rq, rq_batch), sp.nvflat);
                sp.nrq = (sp.nvflat + sp.rq - 1) / sp.rq;
                sp.nfin = sp.nxb * sp.nrq;
                sp.fin_base = fin_base;
                fin_base += sp.nfin;
            }
            c->h.nfin_total = fin_base;
            avl_status st = upload_args(c);
            if (st) {
                std::string m = c->err;
                avl_destroy(b);
                return fail(nullptr, st, m);
            }
        }
    }
    *out = b;
    return AVL_OK;
}

avl_status avl_set_wait_limit(avl_ctx* c, int64_t polls)
{
    if (!c) return AVL_EINVAL;
    const long long wl = polls < 0 ? WAIT_LIMIT : (long long)polls;
    std::vector<avl_ctx*> targets = c->runs.empty() ? std::vector<avl_ctx*>{c} : c->runs;
    for (avl_ctx* t : targets) {
        AVL_CUDA(c, cudaMemcpyAsync(&t->d_ctl->wait_limit, &wl, sizeof(wl), cudaMemcpyHostToDevice, c->st));
        AVL_CUDA(c, cudaStreamSynchronize(c->st));
    }
    return AVL_OK;
}

avl_status avl_batch_run(avl_ctx* b, int32_t r, avl_ctx** run)
{
    if (!b || !run) return AVL_EINVAL;
    if (r < 0 || r >= (int)b->runs.size()) return fail(b, AVL_EINVAL, "run index out of range");
    *run = b->runs[r];
    return AVL_OK;
}

avl_status avl_autotune(avl_ctx* c, int32_t trial_steps, int32_t* chunk_out)
{
    if (!c) return AVL_EINVAL;
    if (trial_steps < 1) return fail(c, AVL_EINVAL, "trial_steps must be >= 1");
    std::vector<avl_ctx*> runs = c->runs;
    if (runs.empty()) runs.push_back(c);
    for (avl_ctx* r : runs)
        if (r->h.nvdim != 1) return fail(c, AVL_EINVAL, "avl_autotune tunes 1d1v contexts");
    // snapshot of every marker set (device), restored after each trial
    struct Snap {
        avl_ctx* r;
        int s;
        long long n;
        double* buf;
    };
    std::vector<Snap> snaps;
    auto release = [&]() {
        for (Snap& q : snaps) cudaFree(q.buf);
        snaps.clear();
    };
    for (avl_ctx* r : runs)
        for (int s = 0; s < r->ns; ++s) {
            if (!r->has_markers[s]) continue;
            Snap q{r, s, r->h.sp[s].n, nullptr};
            cudaError_t e = cudaMalloc(&q.buf, (size_t)q.n * 24);
            if (e) {
                release();
                return cuda_fail(c, e, "cudaMalloc(autotune snapshot)");
            }
            snaps.push_back(q);
            avl_status st = avl_get_markers(r, s, q.buf, q.buf + q.n, q.buf + 2 * q.n, 1);
            if (st) {
                release();
                return fail(c, st, r->err);
            }
        }
    auto restore = [&](int M) -> avl_status {
        for (avl_ctx* r : runs) r->force_M = M;
        for (Snap& q : snaps) {
            avl_status st = avl_set_markers(q.r, q.s, q.n, q.buf, q.buf + q.n, q.buf + 2 * q.n, 1);
            if (st) return fail(c, st, q.r->err);
        }
        return AVL_OK;
    };
    const int cand[] = {0, 1024, 2048, 4096, 8192, 16384};
    int best = 0;
    float best_ms = 0.f;
    cudaEvent_t e0, e1;
    AVL_CUDA(c, cudaEventCreate(&e0));
    AVL_CUDA(c, cudaEventCreate(&e1));
    avl_status st = AVL_OK;
    for (int M : cand) {
        if ((st = restore(M))) break;
        if ((st = avl_step(c, 2))) break;   // builds the step graph
        cudaError_t e = cudaEventRecord(e0, c->st);
        if (!e && (st = avl_step(c, trial_steps))) break;
        if (!e) e = cudaEventRecord(e1, c->st);
        if (!e) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e) {
            st = cuda_fail(c, e, "avl_autotune");
            break;
        }
        if (M == cand[0] || ms < best_ms) {
            best = M;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == AVL_OK) st = restore(best);
    release();
    if (st) return st;
    if (chunk_out) *chunk_out = best;
    return avl_synchronize(c);
}

}  // extern "C"
