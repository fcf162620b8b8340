/*
 * bbmd_oracle.c -- plain FP64 CPU oracle (test infrastructure only; see bbmd_oracle.h).
 *
 * Written from the paper's statement of the method:
 *   Sec. 2.1, Eq. lj0   V(r) = 4 eps_ab [(sigma_ab/r)^12 - (sigma_ab/r)^6]
 *   Sec. 2.1, Eq. sc0   V(r) = 4 eps_ab (sigma_ab/r)^12
 *   Sec. 2.1, Eq. mod0  truncated potential, zero beyond r_c (printed form garbled; read
 *                       as the shifted-force form V - V(rc) - (r-rc) V'(rc); the energy
 *                       shift V - V(rc) and plain truncation are also provided)
 *   Sec. 2.2            O(N) linked-cell search over cubic cells of side >= r_c, with
 *                       Newton's third law halving the pair work
 *   Sec. 2.3.2          velocity-Verlet time marching; forces are the hot spot
 *   Sec. 3              canonical (constant-T) runs: thermostat not named in the paper,
 *                       read as a single Nose-Hoover variable
 *   Sec. 4              radial distribution function g(r)
 *
 * Build: plain C99, -O2 -ffp-contract=off (no fused multiply-add, so every written
 * expression is evaluated as the IEEE operations it shows).
 */
#include "bbmd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------------------------- */
/* pair potential                                                                      */
/* ---------------------------------------------------------------------------------- */

/* Untruncated V(r) and dV/dr of Eq. lj0 / Eq. sc0 at distance r. */
static void raw_pair(const orc_params* p, int a, int b, double r, double* V, double* dV) {
    double eps = p->eps[a][b];
    double sr = p->sigma[a][b] / r;
    double sr6 = sr * sr * sr * sr * sr * sr;
    double sr12 = sr6 * sr6;
    if (p->potential == 0) {
        *V = 4.0 * eps * (sr12 - sr6);
        *dV = 4.0 * eps * (-12.0 * sr12 + 6.0 * sr6) / r;
    } else {
        *V = 4.0 * eps * sr12;
        *dV = 4.0 * eps * (-12.0 * sr12) / r;
    }
}

int orc_pair(const orc_params* p, int a, int b, double r2, double* V, double* f) {
    double rc = p->rcut[a][b];
    if (!(r2 < rc * rc)) {
        *V = 0.0;
        *f = 0.0;
        return 0;
    }
    double r = sqrt(r2);
    double v, dv, vc, dvc;
    raw_pair(p, a, b, r, &v, &dv);
    raw_pair(p, a, b, rc, &vc, &dvc);
    if (p->shift == 0) {          /* plain truncation */
        *V = v;
        *f = -dv / r;
    } else if (p->shift == 1) {   /* energy shift: V - V(rc) */
        *V = v - vc;
        *f = -dv / r;
    } else {                      /* shifted force, Eq. mod0: V - V(rc) - (r - rc) V'(rc) */
        *V = v - vc - (r - rc) * dvc;
        *f = -(dv - dvc) / r;
    }
    return 1;
}

/* plain minimum-image displacement x_j - x_i for wrapped coordinates */
static double min_image(double d, double L) {
    if (d > 0.5 * L)
        d -= L;
    else if (d < -0.5 * L)
        d += L;
    return d;
}

static void zero_outputs(int64_t n, double* F, double* u, double* W, double* PE) {
    if (F) memset(F, 0, sizeof(double) * 3 * (size_t)n);
    if (u) memset(u, 0, sizeof(double) * (size_t)n);
    if (W) *W = 0.0;
    if (PE) *PE = 0.0;
}

/* Accumulate the interaction of pair (i, j) given d = x_j - x_i. */
static void add_pair(int64_t i, int64_t j, const double d[3], const uint8_t* species,
                     const orc_params* p, double* F, double* u, double* W, double* PE) {
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double V, f;
    if (!orc_pair(p, species[i], species[j], r2, &V, &f)) return;
    /* force on i is f * (x_i - x_j) = -f d; Newton's third law gives j the opposite */
    if (F) {
        for (int k = 0; k < 3; ++k) {
            F[3 * i + k] -= f * d[k];
            F[3 * j + k] += f * d[k];
        }
    }
    if (u) {
        u[i] += 0.5 * V;
        u[j] += 0.5 * V;
    }
    if (W) *W += f * r2;
    if (PE) *PE += V;
}

void orc_forces_brute(int64_t n, const double L[3], const uint8_t* species, const double* pos,
                      const orc_params* p, double* F, double* u, double* W, double* PE) {
    zero_outputs(n, F, u, W, PE);
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = i + 1; j < n; ++j) {
            double d[3];
            for (int k = 0; k < 3; ++k) d[k] = min_image(pos[3 * j + k] - pos[3 * i + k], L[k]);
            add_pair(i, j, d, species, p, F, u, W, PE);
        }
    }
}

static double max_rcut(const orc_params* p) {
    double m = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            if (p->rcut[a][b] > m) m = p->rcut[a][b];
    return m;
}

/* Plain cell index of a wrapped coordinate for nc cells over [0, L). */
static int64_t plain_cell(double x, double L, int64_t nc) {
    int64_t c = (int64_t)floor(x / L * (double)nc);
    if (c < 0) c = 0;
    if (c >= nc) c = nc - 1;
    return c;
}

int orc_forces_cells(int64_t n, const double L[3], const uint8_t* species, const double* pos,
                     const orc_params* p, double* F, double* u, double* W, double* PE) {
    double rc = max_rcut(p);
    int64_t nc[3];
    for (int k = 0; k < 3; ++k) {
        nc[k] = (int64_t)floor(L[k] / rc);
        if (nc[k] < 3) return -1;
    }
    int64_t ncell = nc[0] * nc[1] * nc[2];
    int64_t* head = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
    int64_t* next = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t* cidx = (int64_t*)malloc(sizeof(int64_t) * 3 * (size_t)(n > 0 ? n : 1));
    for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
    /* linked list per cell (the paper keeps one list per cell, Sec. 2.2) */
    for (int64_t i = 0; i < n; ++i) {
        for (int k = 0; k < 3; ++k) cidx[3 * i + k] = plain_cell(pos[3 * i + k], L[k], nc[k]);
        int64_t c = (cidx[3 * i + 2] * nc[1] + cidx[3 * i + 1]) * nc[0] + cidx[3 * i];
        next[i] = head[c];
        head[c] = i;
    }
    zero_outputs(n, F, u, W, PE);
    for (int64_t i = 0; i < n; ++i) {
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int64_t ax = (cidx[3 * i] + dx + nc[0]) % nc[0];
                    int64_t ay = (cidx[3 * i + 1] + dy + nc[1]) % nc[1];
                    int64_t az = (cidx[3 * i + 2] + dz + nc[2]) % nc[2];
                    int64_t c = (az * nc[1] + ay) * nc[0] + ax;
                    for (int64_t j = head[c]; j >= 0; j = next[j]) {
                        if (j <= i) continue; /* Newton's third law: each pair once */
                        double d[3];
                        for (int k = 0; k < 3; ++k)
                            d[k] = min_image(pos[3 * j + k] - pos[3 * i + k], L[k]);
                        add_pair(i, j, d, species, p, F, u, W, PE);
                    }
                }
    }
    free(head);
    free(next);
    free(cidx);
    return 0;
}

/* All-core form of the linked-cell forces, for the CPU baseline.  Every particle sums its
 * own 27-cell stencil, so each pair is seen from both ends (a full neighbour set, as on the
 * GPU).  Particles are then independent: the loop over them is shared out over every core
 * (OpenMP), with one writer per force and per u_i.  PE is the serial sum of the u_i. */
int orc_forces_cells_full(int64_t n, const double L[3], const uint8_t* species, const double* pos,
                          const orc_params* p, double* F, double* u, double* PE) {
    double rc = max_rcut(p);
    int64_t nc[3];
    for (int k = 0; k < 3; ++k) {
        nc[k] = (int64_t)floor(L[k] / rc);
        if (nc[k] < 3) return -1;
    }
    int64_t ncell = nc[0] * nc[1] * nc[2];
    int64_t* head = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
    int64_t* next = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t* cidx = (int64_t*)malloc(sizeof(int64_t) * 3 * (size_t)(n > 0 ? n : 1));
    double* ui = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
    for (int64_t i = 0; i < n; ++i) {
        for (int k = 0; k < 3; ++k) cidx[3 * i + k] = plain_cell(pos[3 * i + k], L[k], nc[k]);
        int64_t c = (cidx[3 * i + 2] * nc[1] + cidx[3 * i + 1]) * nc[0] + cidx[3 * i];
        next[i] = head[c];
        head[c] = i;
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double fi[3] = {0.0, 0.0, 0.0}, vi = 0.0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int64_t ax = (cidx[3 * i] + dx + nc[0]) % nc[0];
                    int64_t ay = (cidx[3 * i + 1] + dy + nc[1]) % nc[1];
                    int64_t az = (cidx[3 * i + 2] + dz + nc[2]) % nc[2];
                    int64_t c = (az * nc[1] + ay) * nc[0] + ax;
                    for (int64_t j = head[c]; j >= 0; j = next[j]) {
                        if (j == i) continue;
                        double d[3];
                        for (int k = 0; k < 3; ++k)
                            d[k] = min_image(pos[3 * j + k] - pos[3 * i + k], L[k]);
                        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        double V, f;
                        if (!orc_pair(p, species[i], species[j], r2, &V, &f)) continue;
                        for (int k = 0; k < 3; ++k) fi[k] -= f * d[k];
                        vi += 0.5 * V;
                    }
                }
        if (F)
            for (int k = 0; k < 3; ++k) F[3 * i + k] = fi[k];
        ui[i] = vi;
    }
    double pe = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (u) u[i] = ui[i];
        pe += ui[i];
    }
    if (PE) *PE = pe;
    free(head);
    free(next);
    free(cidx);
    free(ui);
    return 0;
}

/* Threads the all-core form uses (1 when built without OpenMP). */
int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int orc_forces_subset(int64_t n, const double L[3], const uint8_t* species, const double* pos,
                      const orc_params* p, int64_t m, const int64_t* idx, double* F, double* u) {
    double rc = max_rcut(p);
    int64_t nc[3];
    for (int k = 0; k < 3; ++k) {
        nc[k] = (int64_t)floor(L[k] / rc);
        if (nc[k] < 3) return -1;
    }
    int64_t ncell = nc[0] * nc[1] * nc[2];
    int64_t* head = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
    int64_t* next = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
    for (int64_t i = 0; i < n; ++i) {
        int64_t a0 = plain_cell(pos[3 * i], L[0], nc[0]);
        int64_t a1 = plain_cell(pos[3 * i + 1], L[1], nc[1]);
        int64_t a2 = plain_cell(pos[3 * i + 2], L[2], nc[2]);
        int64_t c = (a2 * nc[1] + a1) * nc[0] + a0;
        next[i] = head[c];
        head[c] = i;
    }
    for (int64_t s = 0; s < m; ++s) {
        int64_t i = idx[s];
        double f[3] = {0.0, 0.0, 0.0}, ui = 0.0;
        int64_t a[3];
        for (int k = 0; k < 3; ++k) a[k] = plain_cell(pos[3 * i + k], L[k], nc[k]);
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int64_t bx = (a[0] + dx + nc[0]) % nc[0];
                    int64_t by = (a[1] + dy + nc[1]) % nc[1];
                    int64_t bz = (a[2] + dz + nc[2]) % nc[2];
                    for (int64_t j = head[(bz * nc[1] + by) * nc[0] + bx]; j >= 0; j = next[j]) {
                        if (j == i) continue;
                        double d[3];
                        for (int k = 0; k < 3; ++k)
                            d[k] = min_image(pos[3 * j + k] - pos[3 * i + k], L[k]);
                        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        double V, fr;
                        if (!orc_pair(p, species[i], species[j], r2, &V, &fr)) continue;
                        for (int k = 0; k < 3; ++k) f[k] -= fr * d[k];
                        ui += 0.5 * V;
                    }
                }
        for (int k = 0; k < 3; ++k) F[3 * s + k] = f[k];
        if (u) u[s] = ui;
    }
    free(head);
    free(next);
    return 0;
}

/* ---------------------------------------------------------------------------------- */
/* fixed-point positions, cells, neighbour sets                                        */
/* ---------------------------------------------------------------------------------- */

int orc_fix_exponent(const double L[3]) {
    double m = L[0];
    if (L[1] > m) m = L[1];
    if (L[2] > m) m = L[2];
    if (!(L[0] >= 1.0 && L[1] >= 1.0 && L[2] >= 1.0)) return -1;
    int e;
    frexp(m, &e); /* m = f * 2^e, f in [0.5, 1): floor(log2 m) = e - 1 */
    return 61 - (e - 1);
}

void orc_quantize(int64_t n, const double L[3], int k, const double* pos, int64_t* xfix) {
    for (int d = 0; d < 3; ++d) {
        int64_t Lf = llrint(ldexp(L[d], k));
        for (int64_t i = 0; i < n; ++i) {
            int64_t q = llrint(ldexp(pos[3 * i + d], k));
            q %= Lf;
            if (q < 0) q += Lf;
            xfix[3 * i + d] = q;
        }
    }
}

static int bitlen_u64(uint64_t v) {
    int b = 0;
    while (v) {
        ++b;
        v >>= 1;
    }
    return b;
}

int orc_cell_grid(const double L[3], int k, double rcell, int64_t nc[3], int64_t D[3]) {
    for (int d = 0; d < 3; ++d) {
        int64_t Lf = llrint(ldexp(L[d], k));
        int64_t m = (int64_t)floor(L[d] / rcell);
        for (;;) {
            if (m < 3) return -1;
            uint64_t q = (uint64_t)(Lf / m);
            int bl = bitlen_u64(q);
            if (bl > 24) q &= ~((((uint64_t)1) << (bl - 24)) - 1);
            if (ldexp((double)q, -k) >= rcell) {
                nc[d] = m;
                D[d] = (int64_t)q;
                break;
            }
            --m;
        }
    }
    return 0;
}

void orc_bin(int64_t n, const int64_t* xfix, const int64_t nc[3], const int64_t D[3],
             int64_t* cell) {
    for (int64_t i = 0; i < n; ++i) {
        int64_t a[3];
        for (int d = 0; d < 3; ++d) {
            a[d] = xfix[3 * i + d] / D[d];
            if (a[d] > nc[d] - 1) a[d] = nc[d] - 1;
        }
        cell[i] = (a[2] * nc[1] + a[1]) * nc[0] + a[0];
    }
}

double orc_r2_fixed(const int64_t* xi, const int64_t* xj, const int64_t Lfix[3], int k) {
    double dd[3];
    for (int d = 0; d < 3; ++d) {
        int64_t dx = xj[d] - xi[d];
        if (2 * dx > Lfix[d])
            dx -= Lfix[d];
        else if (2 * dx < -Lfix[d])
            dx += Lfix[d];
        dd[d] = ldexp((double)dx, -k);
    }
    return (dd[0] * dd[0] + dd[1] * dd[1]) + dd[2] * dd[2];
}

static void lfix_of(const double L[3], int k, int64_t Lf[3]) {
    for (int d = 0; d < 3; ++d) Lf[d] = llrint(ldexp(L[d], k));
}

void orc_neighbors_brute(int64_t n, const double L[3], int k, const int64_t* xfix,
                         const uint8_t* species, const double R2[2][2], int64_t* offsets,
                         int64_t* nbr) {
    int64_t Lf[3];
    lfix_of(L, k, Lf);
    int64_t pos = 0;
    for (int64_t i = 0; i < n; ++i) {
        offsets[i] = pos;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double r2 = orc_r2_fixed(xfix + 3 * i, xfix + 3 * j, Lf, k);
            if (r2 < R2[species[i]][species[j]]) {
                if (nbr) nbr[pos] = j;
                ++pos;
            }
        }
    }
    offsets[n] = pos;
}

static int cmp_i64(const void* a, const void* b) {
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x > y) - (x < y);
}

int orc_neighbors_cells(int64_t n, const double L[3], int k, const int64_t* xfix,
                        const uint8_t* species, const double R2[2][2], double rcell,
                        int64_t* offsets, int64_t* nbr) {
    int64_t nc[3], D[3], Lf[3];
    if (orc_cell_grid(L, k, rcell, nc, D) != 0) return -1;
    lfix_of(L, k, Lf);
    int64_t ncell = nc[0] * nc[1] * nc[2];
    int64_t* cell = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t* head = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
    int64_t* next = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    orc_bin(n, xfix, nc, D, cell);
    for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
    for (int64_t i = n - 1; i >= 0; --i) {
        next[i] = head[cell[i]];
        head[cell[i]] = i;
    }
    int64_t pos = 0;
    for (int64_t i = 0; i < n; ++i) {
        offsets[i] = pos;
        int64_t c = cell[i];
        int64_t ax = c % nc[0], ay = (c / nc[0]) % nc[1], az = c / (nc[0] * nc[1]);
        int64_t start = pos;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int64_t bx = (ax + dx + nc[0]) % nc[0];
                    int64_t by = (ay + dy + nc[1]) % nc[1];
                    int64_t bz = (az + dz + nc[2]) % nc[2];
                    int64_t c2 = (bz * nc[1] + by) * nc[0] + bx;
                    for (int64_t j = head[c2]; j >= 0; j = next[j]) {
                        if (j == i) continue;
                        double r2 = orc_r2_fixed(xfix + 3 * i, xfix + 3 * j, Lf, k);
                        if (r2 < R2[species[i]][species[j]]) {
                            if (nbr) nbr[pos] = j;
                            ++pos;
                        }
                    }
                }
        if (nbr) qsort(nbr + start, (size_t)(pos - start), sizeof(int64_t), cmp_i64);
    }
    offsets[n] = pos;
    free(cell);
    free(head);
    free(next);
    return 0;
}

int orc_neighbors_subset(int64_t n, const double L[3], int k, const int64_t* xfix,
                         const uint8_t* species, const double R2[2][2], double rcell, int64_t m,
                         const int64_t* idx, int64_t* offsets, int64_t* nbr) {
    int64_t nc[3], D[3], Lf[3];
    if (orc_cell_grid(L, k, rcell, nc, D) != 0) return -1;
    lfix_of(L, k, Lf);
    int64_t ncell = nc[0] * nc[1] * nc[2];
    int64_t* cell = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t* head = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
    int64_t* next = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    orc_bin(n, xfix, nc, D, cell);
    for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
    for (int64_t i = n - 1; i >= 0; --i) {
        next[i] = head[cell[i]];
        head[cell[i]] = i;
    }
    int64_t pos = 0;
    for (int64_t s = 0; s < m; ++s) {
        int64_t i = idx[s];
        offsets[s] = pos;
        int64_t c = cell[i];
        int64_t ax = c % nc[0], ay = (c / nc[0]) % nc[1], az = c / (nc[0] * nc[1]);
        int64_t start = pos;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int64_t bx = (ax + dx + nc[0]) % nc[0];
                    int64_t by = (ay + dy + nc[1]) % nc[1];
                    int64_t bz = (az + dz + nc[2]) % nc[2];
                    for (int64_t j = head[(bz * nc[1] + by) * nc[0] + bx]; j >= 0; j = next[j]) {
                        if (j == i) continue;
                        double r2 = orc_r2_fixed(xfix + 3 * i, xfix + 3 * j, Lf, k);
                        if (r2 < R2[species[i]][species[j]]) {
                            if (nbr) nbr[pos] = j;
                            ++pos;
                        }
                    }
                }
        if (nbr) qsort(nbr + start, (size_t)(pos - start), sizeof(int64_t), cmp_i64);
    }
    offsets[m] = pos;
    free(cell);
    free(head);
    free(next);
    return 0;
}

/* ---------------------------------------------------------------------------------- */
/* integration                                                                         */
/* ---------------------------------------------------------------------------------- */

double orc_kinetic(int64_t n, const uint8_t* species, const double* vel, const orc_params* p,
                   double P[3]) {
    double K = 0.0;
    double Px = 0.0, Py = 0.0, Pz = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double m = p->mass[species[i]];
        const double* v = vel + 3 * i;
        K += 0.5 * m * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        Px += m * v[0];
        Py += m * v[1];
        Pz += m * v[2];
    }
    if (P) {
        P[0] = Px;
        P[1] = Py;
        P[2] = Pz;
    }
    return K;
}

static int compute_forces(int64_t n, const double L[3], const uint8_t* species,
                          const double* pos, const orc_params* p, double* F, double* PE,
                          int use_cells) {
    if (use_cells == 2) return orc_forces_cells_full(n, L, species, pos, p, F, NULL, PE);
    if (use_cells) return orc_forces_cells(n, L, species, pos, p, F, NULL, NULL, PE);
    orc_forces_brute(n, L, species, pos, p, F, NULL, NULL, PE);
    return 0;
}

/* One Nose-Hoover half step (Trotter split of the thermostat, Martyna-Tuckerman-Klein):
 * xi += dt/4 (2K - gT)/Q; v *= exp(-xi dt/2); eta += xi dt/2; xi += dt/4 (2K' - gT)/Q. */
static void nh_half(int64_t n, const uint8_t* species, double* vel, const orc_params* p,
                    orc_nh* nh, double dt, double T, double tau) {
    double g = (double)(3 * n - 3);
    double Q = g * T * tau * tau;
    double K = orc_kinetic(n, species, vel, p, NULL);
    nh->xi += 0.25 * dt * (2.0 * K - g * T) / Q;
    double s = exp(-nh->xi * 0.5 * dt);
    for (int64_t i = 0; i < 3 * n; ++i) vel[i] *= s;
    nh->eta += nh->xi * 0.5 * dt;
    K = orc_kinetic(n, species, vel, p, NULL);
    nh->xi += 0.25 * dt * (2.0 * K - g * T) / Q;
}

/* wrap into [0, L): x_w = x - L s with s = floor(x/L), s corrected by one when rounding
 * leaves x_w outside [0, L); the crossing count s is added to the image counter */
static void wrap(int64_t n, const double L[3], double* pos, int32_t* image) {
    for (int64_t i = 0; i < n; ++i) {
        for (int d = 0; d < 3; ++d) {
            double x = pos[3 * i + d];
            if (x >= 0.0 && x < L[d]) continue;
            double s = floor(x / L[d]);
            double xw = x - L[d] * s;
            if (xw >= L[d]) {
                xw -= L[d];
                s += 1.0;
            } else if (xw < 0.0) {
                xw += L[d];
                s -= 1.0;
            }
            if (!(xw >= 0.0 && xw < L[d])) xw = 0.0;
            pos[3 * i + d] = xw;
            if (image) image[3 * i + d] += (int32_t)s;
        }
    }
}

int orc_md_run(int64_t n, const double L[3], const uint8_t* species, const orc_params* p,
               double* pos, double* vel, int32_t* image, double* F, int F_valid, orc_nh* nh,
               int64_t nsteps, double dt, const orc_thermo* thermo, int use_cells,
               double* log) {
    int nvt = thermo && thermo->kind == 1;
    double PE = 0.0;
    if (!F_valid && compute_forces(n, L, species, pos, p, F, &PE, use_cells) != 0) return -1;
    for (int64_t s = 0; s < nsteps; ++s) {
        double T = 0.0;
        if (nvt) {
            T = thermo->T_start + (thermo->T_end - thermo->T_start) * (double)s / (double)nsteps;
            nh_half(n, species, vel, p, nh, dt, T, thermo->tau);
        }
        for (int64_t i = 0; i < n; ++i) {
            double h = 0.5 * dt / p->mass[species[i]];
            for (int d = 0; d < 3; ++d) vel[3 * i + d] += F[3 * i + d] * h;
        }
        for (int64_t i = 0; i < 3 * n; ++i) pos[i] += vel[i] * dt;
        wrap(n, L, pos, image);
        if (compute_forces(n, L, species, pos, p, F, &PE, use_cells) != 0) return -1;
        for (int64_t i = 0; i < n; ++i) {
            double h = 0.5 * dt / p->mass[species[i]];
            for (int d = 0; d < 3; ++d) vel[3 * i + d] += F[3 * i + d] * h;
        }
        if (nvt) nh_half(n, species, vel, p, nh, dt, T, thermo->tau);
        if (nh) nh->step += 1;
        if (log) {
            log[5 * s + 0] = orc_kinetic(n, species, vel, p, NULL);
            log[5 * s + 1] = PE;
            log[5 * s + 2] = nh ? nh->xi : 0.0;
            log[5 * s + 3] = nh ? nh->eta : 0.0;
            log[5 * s + 4] = T;
        }
    }
    return 0;
}

int orc_sd_run(int64_t n, const double L[3], const uint8_t* species, const orc_params* p,
               double* pos, int64_t nsteps, double hmax, double dmax, int use_cells) {
    double* F = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    for (int64_t s = 0; s < nsteps; ++s) {
        double PE;
        if (compute_forces(n, L, species, pos, p, F, &PE, use_cells) != 0) {
            free(F);
            return -1;
        }
        double fmax = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double f2 = F[3 * i] * F[3 * i] + F[3 * i + 1] * F[3 * i + 1] + F[3 * i + 2] * F[3 * i + 2];
            double f = sqrt(f2);
            if (f > fmax) fmax = f;
        }
        double h = hmax;
        if (fmax > 0.0 && dmax / fmax < h) h = dmax / fmax;
        for (int64_t i = 0; i < 3 * n; ++i) pos[i] += h * F[i];
        wrap(n, L, pos, NULL);
    }
    free(F);
    return 0;
}

/* ---------------------------------------------------------------------------------- */
/* observables                                                                         */
/* ---------------------------------------------------------------------------------- */

void orc_gr_counts(int64_t n, const double L[3], int k, const int64_t* xfix,
                   const uint8_t* species, int64_t nbins, double rmax, uint64_t* counts) {
    int64_t Lf[3];
    lfix_of(L, k, Lf);
    double dr = rmax / (double)nbins;
    memset(counts, 0, sizeof(uint64_t) * 4 * (size_t)nbins);
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double r2 = orc_r2_fixed(xfix + 3 * i, xfix + 3 * j, Lf, k);
            double r = sqrt(r2);
            double b = floor(r / dr);
            if (b < (double)nbins) counts[(species[i] * 2 + species[j]) * nbins + (int64_t)b] += 1;
        }
    }
}

void orc_gr_normalize(int64_t n, const double L[3], const uint8_t* species, int64_t nbins,
                      double rmax, const uint64_t* counts, double* g) {
    double V = L[0] * L[1] * L[2];
    double Ns[2] = {0.0, 0.0};
    for (int64_t i = 0; i < n; ++i) Ns[species[i]] += 1.0;
    double dr = rmax / (double)nbins;
    const double pi = 3.14159265358979323846;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            double nb = Ns[b] - (a == b ? 1.0 : 0.0);
            for (int64_t q = 0; q < nbins; ++q) {
                double r0 = dr * (double)q, r1 = dr * (double)(q + 1);
                double shell = (4.0 * pi / 3.0) * (r1 * r1 * r1 - r0 * r0 * r0);
                double denom = Ns[a] * nb * shell;
                double c = (double)counts[(a * 2 + b) * nbins + q];
                g[(a * 2 + b) * nbins + q] = denom > 0.0 ? V * c / denom : 0.0;
            }
        }
}

void orc_msd_fs(int64_t n, const double L[3], const uint8_t* species, const double* pos,
                const int32_t* image, const double* pos0, const int32_t* image0, double kvec,
                double msd[2], double fs[2]) {
    double sm[2] = {0.0, 0.0}, sf[2] = {0.0, 0.0}, cnt[2] = {0.0, 0.0};
    for (int64_t i = 0; i < n; ++i) {
        int a = species[i];
        double d2 = 0.0, c = 0.0;
        for (int d = 0; d < 3; ++d) {
            double u = pos[3 * i + d] + L[d] * (double)image[3 * i + d];
            double u0 = pos0[3 * i + d] + L[d] * (double)image0[3 * i + d];
            double du = u - u0;
            d2 += du * du;
            c += cos(kvec * du);
        }
        sm[a] += d2;
        sf[a] += c / 3.0;
        cnt[a] += 1.0;
    }
    for (int a = 0; a < 2; ++a) {
        msd[a] = cnt[a] > 0.0 ? sm[a] / cnt[a] : 0.0;
        fs[a] = cnt[a] > 0.0 ? sf[a] / cnt[a] : 0.0;
    }
}
