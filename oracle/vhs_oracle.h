/*
 * vhs_oracle.h -- plain FP64 CPU oracle of the Vlasov-Hybrid (VHS) time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check of __graft_entry__
 * and the cpu_baseline / reference leg of bench.py may load this library.
 * The product path (the CUDA library behind include/avl.h) never calls it and
 * shares no header, helper or table with it.
 *
 * Every routine is single-threaded, runs in IEEE double precision, and follows
 * the paper's statement of the method in the order the paper gives it:
 *   - phase-space grid, cell-centred values            (Sec. 3.1, Fig. 3)
 *   - cloud-in-cell (area) weights alpha_ij             (Sec. 2, Fig. 1)
 *   - VHS reconstruction f = sum(alpha f_l)/sum(alpha)  (Sec. 2, Eq. 4)
 *   - velocity moment rho = sum_s q_s sum_j f dv        (Sec. 2; Sec. 3.4.2, Eq. 14)
 *   - spectral Poisson solve with sinc softening        (Sec. 3.1, Eq. 5, Eq. 6a-c)
 *   - field gather with the same weights, then push     (Sec. 2, Fig. 2)
 *   - energy / particle-number / entropy diagnostics    (Sec. 3.4.1, Eq. 12, Eq. 13)
 *   - markers: ppc per cell, weighted to f0             (Sec. 2; Sec. 3.1)
 *
 * What pins each routine (and the one that stays unpinned) is listed in the
 * header comment of vhs_oracle.c.
 */
#ifndef VHS_ORACLE_H
#define VHS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Phase-space grid of one species.  x spans [0, L) in nx cells; velocity
 * dimension d spans [vmin[d], vmax[d]) in nv[d] cells.  For nvdim == 1 only
 * index 0 of nv/vmin/vmax is used and nv[1] = nv[2] = 1 is required. */
typedef struct {
    int32_t nvdim;
    int32_t nx;
    double L;
    int32_t nv[3];
    double vmin[3];
    double vmax[3];
} orc_grid;

/* Initial distribution: f0 = sum_b n_b prod_d M(v_d; u_bd, vth_bd)
 *                           * (1 + sum_m amp_m cos(2 pi mode_m x / L + phase_m)) */
typedef struct {
    int32_t nbeam;
    double beam_n[4];
    double beam_u[4][3];
    double beam_vth[4][3];
    int32_t nmode;
    int32_t mode[64];
    double amp[64];
    double phase[64];
} orc_f0;

uint64_t orc_splitmix64(uint64_t seed, uint64_t n);
double orc_jitter_uniform(uint64_t seed, int32_t species, int64_t marker, int32_t dim);

double orc_f0_eval(const orc_f0* p, int32_t nvdim, double L, double x, const double* v);

int64_t orc_marker_count(const orc_grid* g, const int32_t lattice[4]);
int64_t orc_init_markers(const orc_grid* g, const int32_t lattice[4], const orc_f0* p,
                         int32_t species, uint64_t seed, double jitter,
                         double* x, double* v, double* fl);

void orc_reconstruct(const orc_grid* g, int64_t n, const double* x, const double* v,
                     const double* fl, double* num, double* den, double* f);

void orc_moment(const orc_grid* g, double q, const double* f, double* rho);

void orc_poisson(int32_t nx, double L, double cP, int32_t softening,
                 const double* rho, double* E);

void orc_push(const orc_grid* g, int64_t n, double* x, double* v, double qm, double dt,
              const double* E);

/* Boris push with a static background magnetic field B[3] (1d3v; Sec. 3.2:
 * the full Boris push for background magnetic fields): half kick by E along
 * x, rotation about B by the Boris angle 2 atan(|q/m B dt/2|), half kick,
 * then x += v_x dt wrapped into [0, L).  The force is q (E + v x B) in the
 * normalised units of the library (B carries the factor 1/c of CGS). */
void orc_push_boris(const orc_grid* g, int64_t n, double* x, double* v, double qm, double dt,
                    const double* E, const double B[3]);

/* Marker refinement by tracing back to the initial state (Sec. 2: markers of
 * different weight; a phase-space patch that needs more resolution later is
 * traced back to the initial state and given more markers there).  1d1v.
 * New markers sit on a jittered px x pv sub-lattice of every cell of the box
 * [box[0], box[1]) x [box[2], box[3]) (x cells x velocity rows) at the
 * current time, with the jitter recipe of orc_init_markers (stream species,
 * marker m = ((i - box[0]) * (box[3] - box[2]) + (j - box[2])) * ppc + sub).
 * Each is traced back nhist steps by the inverse of the kick-drift step,
 *   x_n = x_{n+1} - v_{n+1} dt (periodic),  v_n = v_{n+1} - (q/m) dt E^n(x_n),
 * with E^n = Ehist[n * nx ...] the field of state n (n = nhist - 1 .. 0), and
 * takes f_l = f0 at the foot.  Writes x, v, fl at the current time and, if not
 * NULL, the feet x0, v0; returns the number of markers. */
int64_t orc_refine_markers(const orc_grid* g, const int32_t box[4], const int32_t lattice[2], const orc_f0* p,
                           int32_t species, uint64_t seed, double jitter, double qm, double dt, int32_t nhist,
                           const double* Ehist, double* x, double* v, double* fl, double* x0, double* v0);

void orc_diag(const orc_grid* g, double m, const double* f, double out[3]);
double orc_field_energy(int32_t nx, double L, double cP, const double* E);

#ifdef __cplusplus
}
#endif
#endif
