/*
 * vhs_oracle.c -- plain FP64 CPU oracle of the Vlasov-Hybrid (VHS) time step.
 *
 * TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load it.  It shares no code,
 * header, table or helper with the CUDA library.
 *
 * Written for a reader checking it against the paper by eye: one marker or one
 * grid point at a time, no blocking, no fusion, no reordering.  Compiled with
 * -ffp-contract=off so that no multiply-add is fused.
 *
 * What pins each routine (tests/test_oracle_pins.py and friends):
 *   orc_splitmix64          SplitMix64 (Steele, Lea & Flood 2014) recomputed
 *                           bit-for-bit by an independent Python integer
 *                           implementation; uniformity statistics.
 *   orc_f0_eval             normalisation: integral over v of one beam is n_b
 *                           (scipy quadrature); perturbation closed form.
 *   orc_init_markers        every marker lies inside its own cell and sub-cell;
 *                           count = cells * ppc; f_l = f0 at the marker.
 *   orc_reconstruct         brute-force rectangle / hyper-box overlap area of
 *                           the marker cloud with every cell (Fig. 1 definition)
 *                           on tiny grids, periodic images in x, dropped edges
 *                           in v; uniform f_l gives f == const; one interior
 *                           marker has sum(alpha) == 1.
 *   orc_moment              midpoint quadrature of a Maxwellian against the
 *                           erf closed form.
 *   orc_poisson             (a) single Fourier modes against the closed form of
 *                           Eq. 6 and of Eq. 5; (b) softened solve equals
 *                           E = -D phi with -Lap3 phi = cP rho solved by a dense
 *                           linear solve (finite-difference reading of Eq. 6);
 *                           constant rho gives E == 0.
 *   orc_push                E == 0: free streaming x + v t mod L; constant E:
 *                           the discrete parabola of kick-drift leapfrog.
 *   orc_diag, field energy  closed forms for a Maxwellian and a single mode.
 *   orc_refine_markers      free streaming f0(x - v t, v); the closed form of
 *                           the inverse step under a uniform field; the feet
 *                           pushed forward by orc_push return the markers.
 *   whole step              linear Landau damping rate and frequency against the
 *                           root of the plasma dispersion function; two-stream
 *                           growth rate; conservation of N and total energy.
 * Parity unpinned: late-time nonlinear trapping amplitudes (figure only in the
 * paper), see the design notes.
 */
#include "vhs_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static const double ORC_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------ */
/* Counter-based random numbers: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014).
 * Output n of the generator seeded with `seed` is the finaliser applied to
 * seed + (n + 1) * golden-gamma.  Used only for the lattice jitter of the
 * marker initialisation, where the draw cannot be passed in from outside. */
uint64_t orc_splitmix64(uint64_t seed, uint64_t n)
{
    uint64_t z = seed + (n + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Uniform double in [0, 1) for (species, marker index, dimension): stream
 * index n = species << 48 | (4 * marker + dim); top 53 bits of the output. */
double orc_jitter_uniform(uint64_t seed, int32_t species, int64_t marker, int32_t dim)
{
    uint64_t n = ((uint64_t)(uint32_t)species << 48) | ((uint64_t)marker * 4u + (uint64_t)dim);
    uint64_t z = orc_splitmix64(seed, n);
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------------ */
/* Initial distribution (Sec. 3.3 species parameters, Eq. 11; Landau test f0
 * Eq. 17 with a cosine): sum of drifting Maxwellian beams times a sum of
 * Fourier density perturbations. */
double orc_f0_eval(const orc_f0* p, int32_t nvdim, double L, double x, const double* v)
{
    double pert = 1.0;
    for (int m = 0; m < p->nmode; ++m) {
        double k = 2.0 * ORC_PI * (double)p->mode[m] / L;
        pert += p->amp[m] * cos(k * x + p->phase[m]);
    }
    double sum = 0.0;
    for (int b = 0; b < p->nbeam; ++b) {
        double g = p->beam_n[b];
        for (int d = 0; d < nvdim; ++d) {
            double vth = p->beam_vth[b][d];
            double t = (v[d] - p->beam_u[b][d]) / vth;
            g *= exp(-0.5 * t * t) / (sqrt(2.0 * ORC_PI) * vth);
        }
        sum += g;
    }
    return sum * pert;
}

static int64_t cells_v(const orc_grid* g)
{
    return (int64_t)g->nv[0] * g->nv[1] * g->nv[2];
}

int64_t orc_marker_count(const orc_grid* g, const int32_t lattice[4])
{
    int64_t ppc = (int64_t)lattice[0] * lattice[1] * lattice[2] * lattice[3];
    return (int64_t)g->nx * cells_v(g) * ppc;
}

/* Marker creation (Sec. 2: same number of markers in every phase-space cell,
 * weights set to reproduce f0; Sec. 3.1: the grid comes first, markers follow).
 * Cell (i, jx, jy, jz) holds a px * pvx * pvy * pvz sub-lattice; sub-lattice
 * point (a, bx, by, bz) sits at the centre of its sub-cell plus a jitter drawn
 * uniformly from [-jitter/2, jitter/2) sub-cells in each dimension.
 * Marker index m = cell_index * ppc + sub_index, both row-major.  The marker
 * value is f0 evaluated at the marker position.
 * x: n values.  v: nvdim * n values, component-major (v[d*n + m]).  fl: n. */
int64_t orc_init_markers(const orc_grid* g, const int32_t lattice[4], const orc_f0* p,
                         int32_t species, uint64_t seed, double jitter,
                         double* x, double* v, double* fl)
{
    const int64_t n = orc_marker_count(g, lattice);
    const int64_t ppc = (int64_t)lattice[0] * lattice[1] * lattice[2] * lattice[3];
    const double dx = g->L / g->nx;
    double dv[3];
    for (int d = 0; d < 3; ++d) dv[d] = (g->vmax[d] - g->vmin[d]) / g->nv[d];

    for (int64_t i = 0; i < g->nx; ++i)
    for (int64_t jx = 0; jx < g->nv[0]; ++jx)
    for (int64_t jy = 0; jy < g->nv[1]; ++jy)
    for (int64_t jz = 0; jz < g->nv[2]; ++jz) {
        int64_t cell = ((i * g->nv[0] + jx) * g->nv[1] + jy) * g->nv[2] + jz;
        int64_t j[3] = {jx, jy, jz};
        for (int64_t a = 0; a < lattice[0]; ++a)
        for (int64_t bx = 0; bx < lattice[1]; ++bx)
        for (int64_t by = 0; by < lattice[2]; ++by)
        for (int64_t bz = 0; bz < lattice[3]; ++bz) {
            int64_t sub = ((a * lattice[1] + bx) * lattice[2] + by) * lattice[3] + bz;
            int64_t m = cell * ppc + sub;
            int64_t b[3] = {bx, by, bz};

            double u0 = orc_jitter_uniform(seed, species, m, 0);
            double jit0 = (u0 - 0.5) * jitter;
            double xm = ((double)i + ((double)a + 0.5 + jit0) / lattice[0]) * dx;

            double vm[3] = {0.0, 0.0, 0.0};
            for (int d = 0; d < g->nvdim; ++d) {
                double ud = orc_jitter_uniform(seed, species, m, d + 1);
                double jit = (ud - 0.5) * jitter;
                vm[d] = g->vmin[d] + ((double)j[d] + ((double)b[d] + 0.5 + jit) / lattice[d + 1]) * dv[d];
            }
            x[m] = xm;
            for (int d = 0; d < g->nvdim; ++d) v[(int64_t)d * n + m] = vm[d];
            fl[m] = orc_f0_eval(p, g->nvdim, g->L, xm, vm);
        }
    }
    return n;
}

/* ------------------------------------------------------------------------ */
/* One-dimensional cloud-in-cell weights on a cell-centred grid (Fig. 1,
 * Fig. 3): the cloud [y - h/2, y + h/2) overlaps the two cells whose centres
 * bracket y.  u = y/h - 1/2, i0 = floor(u), weight (1 - w) on cell i0 and w on
 * cell i0 + 1, w = u - i0. */
static void cic1(double y_over_h, int64_t* i0, double* w)
{
    double u = y_over_h - 0.5;
    double fl = floor(u);
    *i0 = (int64_t)fl;
    *w = u - fl;
}

/* VHS reconstruction (Sec. 2, Eq. 4): every marker adds alpha * f_l to the
 * numerator and alpha to the denominator of each cell its cloud overlaps,
 * alpha being the overlap fraction (product of 1-D weights); x is periodic,
 * cells beyond the velocity grid are dropped; f = num / den where den > 0,
 * and 0 in cells no marker reaches.  num, den, f: nx * prod(nv) values in
 * row-major [x][vx][vy][vz] order.  num/den may be NULL. */
void orc_reconstruct(const orc_grid* g, int64_t n, const double* x, const double* v,
                     const double* fl, double* num_out, double* den_out, double* f)
{
    const int64_t nvc = cells_v(g);
    const int64_t ncell = (int64_t)g->nx * nvc;
    double* num = (double*)calloc((size_t)ncell, sizeof(double));
    double* den = (double*)calloc((size_t)ncell, sizeof(double));
    const double dx = g->L / g->nx;
    double dv[3];
    for (int d = 0; d < 3; ++d) dv[d] = (g->vmax[d] - g->vmin[d]) / g->nv[d];

    const int ncorner = 1 << (1 + g->nvdim);
    for (int64_t l = 0; l < n; ++l) {
        int64_t ix0; double wx;
        cic1(x[l] / dx, &ix0, &wx);
        int64_t jv0[3] = {0, 0, 0};
        double wv[3] = {0.0, 0.0, 0.0};
        for (int d = 0; d < g->nvdim; ++d)
            cic1((v[(int64_t)d * n + l] - g->vmin[d]) / dv[d], &jv0[d], &wv[d]);

        for (int c = 0; c < ncorner; ++c) {
            int cx = c & 1;
            int64_t ix = ix0 + cx;
            ix = ((ix % g->nx) + g->nx) % g->nx;
            double alpha = cx ? wx : 1.0 - wx;
            int64_t jj[3] = {0, 0, 0};
            int inside = 1;
            for (int d = 0; d < g->nvdim; ++d) {
                int cd = (c >> (1 + d)) & 1;
                jj[d] = jv0[d] + cd;
                if (jj[d] < 0 || jj[d] >= g->nv[d]) inside = 0;
                alpha *= cd ? wv[d] : 1.0 - wv[d];
            }
            if (!inside) continue;
            int64_t cell = ((ix * g->nv[0] + jj[0]) * g->nv[1] + jj[1]) * g->nv[2] + jj[2];
            num[cell] += alpha * fl[l];
            den[cell] += alpha;
        }
    }
    for (int64_t c = 0; c < ncell; ++c) {
        f[c] = den[c] > 0.0 ? num[c] / den[c] : 0.0;
        if (num_out) num_out[c] = num[c];
        if (den_out) den_out[c] = den[c];
    }
    free(num);
    free(den);
}

/* Velocity moment (Sec. 2; Eq. 14): rho_i += q * prod(dv) * sum_j f_ij,
 * midpoint rule over the cell-centred velocity grid, no interpolation. */
void orc_moment(const orc_grid* g, double q, const double* f, double* rho)
{
    const int64_t nvc = cells_v(g);
    double dvol = 1.0;
    for (int d = 0; d < g->nvdim; ++d) dvol *= (g->vmax[d] - g->vmin[d]) / g->nv[d];
    for (int64_t i = 0; i < g->nx; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < nvc; ++j) s += f[i * nvc + j];
        rho[i] += q * dvol * s;
    }
}

/* Spectral Poisson solve (Sec. 3.1, Eq. 5 and Eq. 6a-c), by a plain discrete
 * Fourier transform: rho_hat_m = sum_i rho_i exp(-2 pi i m i / N);
 * E_hat_m = -i cP kappa_m / K2_m rho_hat_m with, when softening is on,
 * kappa = k sinc(k dx), K2 = k^2 sinc^2(k dx / 2), sinc(y) = sin(y)/y, and
 * kappa = k, K2 = k^2 otherwise; k_m = 2 pi m' / L with m' the signed mode
 * number.  The k = 0 mode is removed (neutralising background) and the
 * Nyquist mode of an even N is set to zero.  E_i = (1/N) sum_m E_hat_m
 * exp(+2 pi i m i / N). */
void orc_poisson(int32_t nx, double L, double cP, int32_t softening,
                 const double* rho, double* E)
{
    const int64_t N = nx;
    const double dx = L / (double)N;
    double* er = (double*)calloc((size_t)N, sizeof(double));
    double* ei = (double*)calloc((size_t)N, sizeof(double));
    for (int64_t m = 0; m < N; ++m) {
        if (m == 0 || 2 * m == N) continue;
        double rr = 0.0, ri = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            double ang = 2.0 * ORC_PI * (double)((m * i) % N) / (double)N;
            rr += rho[i] * cos(ang);
            ri -= rho[i] * sin(ang);
        }
        int64_t ms = (2 * m < N) ? m : m - N;
        double k = 2.0 * ORC_PI * (double)ms / L;
        double kappa, K2;
        if (softening) {
            double y1 = k * dx, y2 = 0.5 * k * dx;
            kappa = k * (sin(y1) / y1);
            K2 = k * k * (sin(y2) / y2) * (sin(y2) / y2);
        } else {
            kappa = k;
            K2 = k * k;
        }
        double gm = cP * kappa / K2;
        /* -i * gm * (rr + i ri) = gm * ri - i gm * rr */
        er[m] = gm * ri;
        ei[m] = -gm * rr;
    }
    for (int64_t i = 0; i < N; ++i) {
        double s = 0.0;
        for (int64_t m = 0; m < N; ++m) {
            double ang = 2.0 * ORC_PI * (double)((m * i) % N) / (double)N;
            s += er[m] * cos(ang) - ei[m] * sin(ang);
        }
        E[i] = s / (double)N;
    }
    free(er);
    free(ei);
}

/* Marker push (Sec. 2, Fig. 2): the grid field is interpolated to the marker
 * with the same cloud-in-cell x-weights as the reconstruction; then the
 * velocity is kicked, v += (q/m) E dt, and the position drifts with the new
 * velocity, x += v dt, wrapped into [0, L).  Only v_x feels the field (no
 * magnetic field), v_y and v_z ride along unchanged. */
void orc_push(const orc_grid* g, int64_t n, double* x, double* v, double qm, double dt,
              const double* E)
{
    const double dx = g->L / g->nx;
    for (int64_t l = 0; l < n; ++l) {
        int64_t i0; double w;
        cic1(x[l] / dx, &i0, &w);
        int64_t ia = ((i0 % g->nx) + g->nx) % g->nx;
        int64_t ib = (((i0 + 1) % g->nx) + g->nx) % g->nx;
        double El = (1.0 - w) * E[ia] + w * E[ib];
        double vx = v[l] + qm * El * dt;
        double xn = x[l] + vx * dt;
        xn = fmod(xn, g->L);
        if (xn < 0.0) xn += g->L;
        if (xn >= g->L) xn -= g->L;
        v[l] = vx;
        x[l] = xn;
    }
}

/* Boris push (Boris 1970; Birdsall & Langdon Sec. 4-4): with a = (q/m) dt/2,
 * v- = v + a E x_hat; t = a B; s = 2 t / (1 + |t|^2);
 * v' = v- + v- x t;  v+ = v- + v' x s;  v_new = v+ + a E x_hat;
 * x_new = x + v_new,x dt (periodic).  E is gathered with the cloud-in-cell
 * weights of the reconstruction, as in orc_push.  v is component-major
 * (v[d * n + l]). */
void orc_push_boris(const orc_grid* g, int64_t n, double* x, double* v, double qm, double dt,
                    const double* E, const double B[3])
{
    const double dx = g->L / g->nx;
    const double a = 0.5 * qm * dt;
    const double t[3] = {a * B[0], a * B[1], a * B[2]};
    const double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    const double sf = 2.0 / (1.0 + t2);
    const double s[3] = {sf * t[0], sf * t[1], sf * t[2]};
    for (int64_t l = 0; l < n; ++l) {
        int64_t i0;
        double w;
        cic1(x[l] / dx, &i0, &w);
        int64_t ia = ((i0 % g->nx) + g->nx) % g->nx;
        int64_t ib = (((i0 + 1) % g->nx) + g->nx) % g->nx;
        double El = (1.0 - w) * E[ia] + w * E[ib];
        double vm[3] = {v[l] + a * El, v[n + l], v[2 * n + l]};
        double vp[3] = {vm[0] + (vm[1] * t[2] - vm[2] * t[1]), vm[1] + (vm[2] * t[0] - vm[0] * t[2]),
                        vm[2] + (vm[0] * t[1] - vm[1] * t[0])};
        double vq[3] = {vm[0] + (vp[1] * s[2] - vp[2] * s[1]), vm[1] + (vp[2] * s[0] - vp[0] * s[2]),
                        vm[2] + (vp[0] * s[1] - vp[1] * s[0])};
        double vx = vq[0] + a * El;
        double xn = x[l] + vx * dt;
        xn = fmod(xn, g->L);
        if (xn < 0.0) xn += g->L;
        if (xn >= g->L) xn -= g->L;
        v[l] = vx;
        v[n + l] = vq[1];
        v[2 * n + l] = vq[2];
        x[l] = xn;
    }
}

/* Marker refinement by tracing back (Sec. 2), see the header. */
int64_t orc_refine_markers(const orc_grid* g, const int32_t box[4], const int32_t lattice[2], const orc_f0* p,
                           int32_t species, uint64_t seed, double jitter, double qm, double dt, int32_t nhist,
                           const double* Ehist, double* x, double* v, double* fl, double* x0, double* v0)
{
    const double dx = g->L / g->nx;
    const double dv = (g->vmax[0] - g->vmin[0]) / g->nv[0];
    const int64_t ppc = (int64_t)lattice[0] * lattice[1];
    const int64_t nrow = box[3] - box[2];
    int64_t m = 0;
    for (int64_t i = box[0]; i < box[1]; ++i)
    for (int64_t j = box[2]; j < box[3]; ++j)
    for (int64_t a = 0; a < lattice[0]; ++a)
    for (int64_t b = 0; b < lattice[1]; ++b) {
        m = ((i - box[0]) * nrow + (j - box[2])) * ppc + a * lattice[1] + b;
        double jx = (orc_jitter_uniform(seed, species, m, 0) - 0.5) * jitter;
        double jv = (orc_jitter_uniform(seed, species, m, 1) - 0.5) * jitter;
        double xm = ((double)i + ((double)a + 0.5 + jx) / lattice[0]) * dx;
        double vm = g->vmin[0] + ((double)j + ((double)b + 0.5 + jv) / lattice[1]) * dv;
        x[m] = xm;
        v[m] = vm;
        /* back along the characteristic: undo the drift, then the kick of
         * state n, whose field is gathered at the earlier position */
        for (int32_t n = nhist - 1; n >= 0; --n) {
            double xn = xm - vm * dt;
            xn = fmod(xn, g->L);
            if (xn < 0.0) xn += g->L;
            if (xn >= g->L) xn -= g->L;
            xm = xn;
            int64_t i0; double w;
            cic1(xm / dx, &i0, &w);
            int64_t ia = ((i0 % g->nx) + g->nx) % g->nx;
            int64_t ib = (((i0 + 1) % g->nx) + g->nx) % g->nx;
            const double* E = Ehist + (int64_t)n * g->nx;
            double El = (1.0 - w) * E[ia] + w * E[ib];
            vm = vm - qm * El * dt;
        }
        if (x0) x0[m] = xm;
        if (v0) v0[m] = vm;
        fl[m] = orc_f0_eval(p, 1, g->L, xm, &vm);
    }
    return (box[1] - box[0]) * nrow * ppc;
}

/* Diagnostics of one species on its reconstructed grid (Sec. 3.4.1):
 * out[0] = N = sum f dx dv                       (number of particles)
 * out[1] = W_kin = m/2 sum |v_j|^2 f dx dv        (kinetic energy, cell centres)
 * out[2] = S = sum_{f>0} f log f dx dv           (Eq. 13, coarse-grained entropy) */
void orc_diag(const orc_grid* g, double m, const double* f, double out[3])
{
    const int64_t nvc = cells_v(g);
    const double dx = g->L / g->nx;
    double dv[3] = {1.0, 1.0, 1.0};
    double dvol = 1.0;
    for (int d = 0; d < g->nvdim; ++d) {
        dv[d] = (g->vmax[d] - g->vmin[d]) / g->nv[d];
        dvol *= dv[d];
    }
    double N = 0.0, W = 0.0, S = 0.0;
    for (int64_t i = 0; i < g->nx; ++i)
    for (int64_t jx = 0; jx < g->nv[0]; ++jx)
    for (int64_t jy = 0; jy < g->nv[1]; ++jy)
    for (int64_t jz = 0; jz < g->nv[2]; ++jz) {
        double fv = f[((i * g->nv[0] + jx) * g->nv[1] + jy) * g->nv[2] + jz];
        int64_t j[3] = {jx, jy, jz};
        double v2 = 0.0;
        for (int d = 0; d < g->nvdim; ++d) {
            double vc = g->vmin[d] + ((double)j[d] + 0.5) * dv[d];
            v2 += vc * vc;
        }
        N += fv;
        W += v2 * fv;
        if (fv > 0.0) S += fv * log(fv);
    }
    out[0] = N * dx * dvol;
    out[1] = 0.5 * m * W * dx * dvol;
    out[2] = S * dx * dvol;
}

/* Field energy (Eq. 12 read for one dimension): W_E = 1/(2 cP) sum_i E_i^2 dx;
 * cP = 4 pi gives the paper's 1/(8 pi). */
double orc_field_energy(int32_t nx, double L, double cP, const double* E)
{
    double s = 0.0;
    for (int32_t i = 0; i < nx; ++i) s += E[i] * E[i];
    return s * (L / nx) / (2.0 * cP);
}
