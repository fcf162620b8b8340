/*
 * bbmd_oracle.h -- plain, slow FP64 CPU oracle for the short-range molecular-dynamics
 * method of Allsopp, Ruocco & Fratalocchi (BBMD, arXiv:1105.5613).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link or call
 * this code: only the test-suite, the smoke check and the benchmark's CPU-baseline
 * leg do.  It shares no code, header, table or constant generator with the CUDA
 * library; both implement the same written definitions.
 *
 * Array conventions: positions, velocities and forces are row-major (n, 3) doubles;
 * species are uint8 labels 0 (A) / 1 (B); pair tables are [2][2] row-major.
 *
 * Parity pins (the tests that tie each function to something other than itself):
 *   orc_pair            dimer minimum -eps at 2^(1/6) sigma, force = -dV/dr by
 *                       Richardson finite differences, V*(rc)=0 and F*(rc)=0 (Eq. mod0)
 *   orc_forces_brute    FCC lattice shell sum (coordination 12,6,24,12,24,...), zero
 *                       lattice forces, Newton's third law, translation invariance
 *   orc_forces_cells    equals orc_forces_brute (paper's search vs the O(N^2) definition)
 *   orc_forces_cells_full  equals orc_forces_brute (all-core full-stencil form)
 *   orc_bin / orc_neighbors_*   brute-force set definition, symmetry, containment
 *   orc_md_run          time reversibility, dt^2 energy-error scaling, momentum,
 *                       Nose-Hoover free-gas ODE (scipy), extended-energy conservation
 *   orc_gr_counts       scipy pdist + histogram on points away from bin edges, totals
 *   orc_msd_fs          rigid translation closed form, t=0 values
 */
#ifndef BBMD_ORACLE_H
#define BBMD_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t potential;   /* 0: Lennard-Jones (Eq. lj0); 1: soft sphere (Eq. sc0)            */
    int32_t shift;       /* 0: plain truncation; 1: energy shift; 2: shifted force (Eq. mod0) */
    double eps[2][2];
    double sigma[2][2];
    double rcut[2][2];
    double mass[2];
} orc_params;

typedef struct {
    int32_t kind;        /* 0: NVE, 1: Nose-Hoover                                          */
    double T_start;      /* target temperature at the first step of the run                 */
    double T_end;        /* target at the end; linear ramp T_k = T_start+(T_end-T_start)k/n  */
    double tau;          /* thermostat time: Q = g T tau^2                                   */
} orc_thermo;

typedef struct {
    double xi;           /* Nose-Hoover friction variable                                   */
    double eta;          /* time integral of xi                                             */
    int64_t step;        /* steps taken                                                     */
} orc_nh;

/* ---- pair potential (Sec. 2.1) ------------------------------------------------------ */
/* V*(r) and f = -(dV*(r)/dr)/r for species a,b at squared distance r2 < rcut^2; returns 1 if
 * the pair interacts (r2 < rcut_ab^2), else 0 with V=f=0. */
int orc_pair(const orc_params* p, int a, int b, double r2, double* V, double* f);

/* ---- forces (Sec. 2.1-2.2) ---------------------------------------------------------- */
/* O(N^2) definition, minimum image (requires rcut < L/2).  F: (n,3); u: per-particle
 * potential energy (half of each pair energy); *W = sum over pairs of r_ij . F_ij;
 * *PE = sum over pairs of V*.  Any output pointer may be NULL. */
void orc_forces_brute(int64_t n, const double L[3], const uint8_t* species, const double* pos,
                      const orc_params* p, double* F, double* u, double* W, double* PE);
/* The paper's linked-cell search with Newton's third law (Sec. 2.2): cells of side >=
 * max rcut, 27-cell stencil, each unordered pair once.  Same outputs.  Returns 0, or -1
 * when the box holds fewer than 3 cells per axis. */
int orc_forces_cells(int64_t n, const double L[3], const uint8_t* species, const double* pos,
                     const orc_params* p, double* F, double* u, double* W, double* PE);

/* The same forces, per-particle energies and PE for the all-core CPU baseline: each
 * particle sums its own 27-cell stencil (each pair seen from both ends), the particles
 * shared out over every core.  -1 if the box holds fewer than 3 cells per axis. */
int orc_forces_cells_full(int64_t n, const double L[3], const uint8_t* species, const double* pos,
                          const orc_params* p, double* F, double* u, double* PE);

/* Threads orc_forces_cells_full uses (1 when built without OpenMP). */
int orc_threads(void);

/* Forces, per-particle energy and virial share of the m particles idx[] only, by the
 * linked-cell search of Sec. 2.2 (both members of every pair visited, no Newton's third
 * law): F[3m], u[m] (may be NULL).  For spot checks of very large systems.  Returns -1
 * when the box holds fewer than 3 cells per axis. */
int orc_forces_subset(int64_t n, const double L[3], const uint8_t* species, const double* pos,
                      const orc_params* p, int64_t m, const int64_t* idx, double* F, double* u);

/* ---- fixed-point positions, cells and neighbour sets --------------------------------- */
/* Unit exponent k: positions are held as integers in units of 2^-k, k = 61 - floor(log2
 * max L).  Returns -1 if some L < 1. */
int orc_fix_exponent(const double L[3]);
/* x_fix = round-half-even(x * 2^k) reduced modulo L*2^k into [0, L*2^k). */
void orc_quantize(int64_t n, const double L[3], int k, const double* pos, int64_t* xfix);
/* Cell grid for cell side >= rcell: nc[d] = floor(L[d]/rcell), D[d] = floor(L_fix/nc)
 * truncated to 24 significant bits (lowered by one cell while D*2^-k < rcell).
 * Returns -1 if some nc < 3. */
int orc_cell_grid(const double L[3], int k, double rcell, int64_t nc[3], int64_t D[3]);
/* cell[i] = (az*ncy + ay)*ncx + ax with a = min(nc-1, x_fix / D). */
void orc_bin(int64_t n, const int64_t* xfix, const int64_t nc[3], const int64_t D[3],
             int64_t* cell);
/* Exact squared distance rule: dx = x_j - x_i as an integer, reduced to the minimum image
 * (|dx| <= L_fix/2), rounded once to double, scaled by 2^-k; r2 = (dx*dx+dy*dy)+dz*dz. */
double orc_r2_fixed(const int64_t* xi, const int64_t* xj, const int64_t Lfix[3], int k);
/* Full neighbour sets {j != i : r2 < R2[s_i][s_j]} by brute force.  offsets: n+1 entries;
 * nbr: ascending j per i.  Pass nbr=NULL to get the counts (offsets) only. */
void orc_neighbors_brute(int64_t n, const double L[3], int k, const int64_t* xfix,
                         const uint8_t* species, const double R2[2][2],
                         int64_t* offsets, int64_t* nbr);
/* Same sets through the cell grid (orc_cell_grid with rcell >= sqrt(max R2)). */
int orc_neighbors_cells(int64_t n, const double L[3], int k, const int64_t* xfix,
                        const uint8_t* species, const double R2[2][2], double rcell,
                        int64_t* offsets, int64_t* nbr);

/* Neighbour sets of the m particles idx[] only (exact rule, cell grid with rcell). */
int orc_neighbors_subset(int64_t n, const double L[3], int k, const int64_t* xfix,
                         const uint8_t* species, const double R2[2][2], double rcell, int64_t m,
                         const int64_t* idx, int64_t* offsets, int64_t* nbr);

/* ---- integration (Sec. 2.3.2, velocity Verlet; canonical runs, Sec. 3) ------------- */
/* Kinetic energy sum m v^2 / 2 and momentum sum m v. */
double orc_kinetic(int64_t n, const uint8_t* species, const double* vel, const orc_params* p,
                   double P[3]);
/* nsteps of velocity Verlet (thermo NULL or kind 0: NVE; kind 1: Nose-Hoover by the
 * splitting NH-half, kick, drift, force, kick, NH-half).  pos is wrapped into [0,L)
 * every step and image[3n] counts the box crossings.  F holds the forces of pos on
 * entry (computed if F_valid == 0) and on exit.  Forces by brute force when
 * use_cells == 0, by orc_forces_cells when 1, by orc_forces_cells_full (every core) when
 * 2.  If log is non-NULL it receives per step
 * {KE, PE, xi, eta, T_target} (5 doubles). */
int orc_md_run(int64_t n, const double L[3], const uint8_t* species, const orc_params* p,
               double* pos, double* vel, int32_t* image, double* F, int F_valid,
               orc_nh* nh, int64_t nsteps, double dt, const orc_thermo* thermo,
               int use_cells, double* log);

/* Steepest descent x += h F with h = min(hmax, dmax / max_i |F_i|), nsteps times. */
int orc_sd_run(int64_t n, const double L[3], const uint8_t* species, const orc_params* p,
               double* pos, int64_t nsteps, double hmax, double dmax, int use_cells);

/* ---- observables (Sec. 4, Eq. for g(r)) -------------------------------------------- */
/* Ordered-pair counts per species pair: counts[(a*2+b)*nbins + bin], bin = floor(r/dr),
 * dr = rmax/nbins, r = sqrt of the exact r2 rule, j != i, bin < nbins. */
void orc_gr_counts(int64_t n, const double L[3], int k, const int64_t* xfix,
                   const uint8_t* species, int64_t nbins, double rmax, uint64_t* counts);
/* g_ab(bin) = V n_ab / (N_a N'_b (4pi/3)(r_{k+1}^3 - r_k^3)), N'_b = N_b - (a==b). */
void orc_gr_normalize(int64_t n, const double L[3], const uint8_t* species, int64_t nbins,
                      double rmax, const uint64_t* counts, double* g);
/* Unwrapped u = x + L*image.  msd[a] = <|u-u0|^2>_a, fs[a] = <(1/3) sum_d cos(k du_d)>_a. */
void orc_msd_fs(int64_t n, const double L[3], const uint8_t* species, const double* pos,
                const int32_t* image, const double* pos0, const int32_t* image0, double kvec,
                double msd[2], double fs[2]);

#ifdef __cplusplus
}
#endif
#endif
