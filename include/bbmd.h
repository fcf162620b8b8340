/*
 * bbmd.h -- C ABI of the GB300 hot path of the short-range molecular-dynamics method of
 * Allsopp, Ruocco & Fratalocchi (BBMD): cell binning, Verlet neighbour list, truncated
 * Lennard-Jones / soft-sphere pair forces of a two-species mixture in a periodic box,
 * velocity Verlet with an optional Nose-Hoover thermostat, device reductions and the
 * observables of the paper's glass study.
 *
 * The paper defines the problem, not an API (Sec. 2.1 potentials, Sec. 2.2 cell search,
 * Sec. 2.3.2 velocity Verlet, Sec. 3 canonical benchmark runs, Sec. 4 g(r)); these calls
 * follow that statement of the problem.
 *
 * Conventions for every call
 *   - Host arrays are caller-owned and only read or written during the call.  Positions,
 *     velocities and forces on the host are row-major (n, 3) doubles in particle-id order
 *     (id = index in the arrays given to bbmd_create).  Species labels are uint8 0 (A)
 *     or 1 (B).
 *   - Device memory is owned by the handle and obtained through the caller's allocator
 *     (bbmd_alloc) or cudaMalloc when it is NULL; bbmd_destroy returns all of it.
 *   - Work is enqueued on the CUDA stream given to bbmd_create (NULL = one owned by the
 *     handle).
 *     bbmd_step returns after enqueueing; every call that returns host data synchronises
 *     that stream.
 *   - Errors are returned as bbmd_status codes, never by abort or exit.  A device-side
 *     status word (staged-stencil overflow, a list beyond 4096 entries, non-finite force,
 *     velocity overflow, a bounded wait that gave up) is sticky and is reported by the
 *     next synchronising call; lists longer than their capacity are grown there instead
 *     (see list_capacity).  bbmd_last_error gives a message.
 *   - A handle is not thread-safe.
 *
 * State representation (the exact rules the test oracle implements independently)
 *   - Positions are held as signed 64-bit integers in units of 2^-k with
 *     k = 61 - floor(log2(max box side)); box sides must be >= 1 and are exact integers
 *     in that unit.  Input positions are quantised as round-half-even(x * 2^k) and
 *     reduced modulo the box into [0, L).  Velocities are 64-bit integers in units of
 *     2^-52 (|v| < 2048).
 *   - Cells: nc = floor(L / rcell) per axis, side D = floor(L*2^k / nc) truncated to 24
 *     significant bits (nc lowered while D*2^-k < rcell); cell a = min(nc-1, x_fix / D).
 *     rcell = max rcut + skin.  Fewer than 3 cells on an axis -> BBMD_ERR_BOX_TOO_SMALL.
 *   - Pair distance: dx = x_j - x_i as an integer, reduced to the minimum image, rounded
 *     once to double, scaled by 2^-k; r^2 = (dx*dx + dy*dy) + dz*dz in IEEE double with
 *     no fused multiply-add.  Cutoff and list decisions use this r^2 with strict "<":
 *     a pair interacts iff r^2 < rcut_ab^2; j is in the Verlet list of i iff
 *     r^2 < (rcut_ab + skin)^2.  Mixed precision evaluates r^2 in FP32 and re-tests in
 *     FP64 by this rule whenever it lies within a relative 1e-5 of the threshold, so
 *     both decisions are exact.
 */
#ifndef BBMD_H
#define BBMD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BBMD_OK = 0,
    BBMD_ERR_ARG = 1,             /* invalid argument                                       */
    BBMD_ERR_BOX_TOO_SMALL = 2,   /* fewer than 3 cells per axis                            */
    BBMD_ERR_OOM = 3,             /* the allocator returned NULL                            */
    BBMD_ERR_CUDA = 4,            /* a CUDA runtime call failed                             */
    BBMD_ERR_LIST_OVERFLOW = 5,   /* a staged stencil, or a list beyond 4096, overflowed    */
    BBMD_ERR_NUMERIC = 6,         /* non-finite force or |v| beyond the fixed-point range   */
    BBMD_ERR_TIMEOUT = 7,         /* a bounded device wait gave up                          */
    BBMD_ERR_STATE = 8            /* call not valid in the handle's current state           */
} bbmd_status;

enum { BBMD_POT_LJ = 0, BBMD_POT_SOFT = 1 };                 /* Eq. lj0, Eq. sc0          */
enum { BBMD_SHIFT_NONE = 0, BBMD_SHIFT_ENERGY = 1,            /* plain cut; V - V(rc)      */
       BBMD_SHIFT_FORCE = 2 };                                /* Eq. mod0 (shifted force)  */
enum { BBMD_PREC_MIXED = 0, BBMD_PREC_FP64 = 1 };             /* FP32 pair math / FP64     */
enum { BBMD_NBR_VERLET = 0, BBMD_NBR_CELL = 1 };              /* stored list / on the fly  */
enum { BBMD_THERMO_NVE = 0, BBMD_THERMO_NH = 1 };

/* Pair model and neighbour-search parameters.
 * eps, sigma, rcut: [a][b] tables (must be symmetric); mass[a] > 0.
 * skin: Verlet skin (>= 0); the list is rebuilt when some particle has moved more than
 *   skin/2 since the last build (Verlet mode) or, in cell mode, when it has left the
 *   margin skin/2 that the cells carry.
 * list_capacity: initial list entries per particle (0 = 160; rounded up to 8).  A build
 *   whose longest list exceeds it keeps going exactly: until the lists are rebuilt, each
 *   step takes its forces from the cell stencil instead.  The next synchronising call
 *   (creation, observe, get_state, set_state, get_forces, get_neighbors, ...) grows the
 *   capacity to the longest list plus an eighth and rebuilds the lists.  Only a list
 *   longer than 4096 entries is reported, as BBMD_ERR_LIST_OVERFLOW.
 * stencil_capacity: maximum particles staged for one block of cells, i.e. in the cells
 *   around it (one layer on every side; 0 = from the density, with 15 % headroom).
 * block_z: block shape code of the force and list kernels, one CTA per block at a time:
 *   1, 2 or 4 = blocks of 2 x 2 x block_z cells; 8 = blocks of 4 x 4 x 2 cells (32 cells);
 *   0 = chosen at creation by timing every shape that fits on the initial state.  (Every
 *   shape keeps its cells within 2 cells of the block's middle, so the FP32 coordinates of
 *   mixed precision stay within 3 cells of their frame.)
 * init_jitter: with pos == NULL (device-generated FCC lattice), coordinate d of site i is
 *   moved by init_jitter * (2u - 1), u = uniform01(draw 3i + d of stream 5) under the
 *   creation seed (0 = the perfect lattice); the displaced position is quantised and
 *   reduced into the box like any input position. */
typedef struct {
    int32_t potential;
    int32_t shift;
    int32_t precision;
    int32_t nbr_mode;
    double eps[2][2];
    double sigma[2][2];
    double rcut[2][2];
    double mass[2];
    double skin;
    int32_t list_capacity;
    int32_t stencil_capacity;
    int32_t block_z;
    double init_jitter;
} bbmd_params;

/* Thermostat of one bbmd_step call.  NVE, or Nose-Hoover with one friction variable xi,
 * Q = g T tau^2 (g = 3n - 3), target T_k = T_start + (T_end - T_start) * k / nsteps for
 * step k = 0 .. nsteps-1 of the call (a linear ramp; constant when T_start == T_end).
 * Each step is NH-half, kick, drift, force, kick, NH-half (Trotter splitting). */
typedef struct {
    int32_t kind;
    double T_start;
    double T_end;
    double tau;
} bbmd_thermostat;

/* Device allocator: alloc returns a device pointer (NULL on failure); free releases it. */
typedef struct {
    void* (*alloc)(size_t bytes, void* ctx);
    void (*free)(void* ptr, void* ctx);
    void* ctx;
} bbmd_alloc;

typedef struct bbmd_sim bbmd_sim;

/* bbmd_observe mask bits */
enum {
    BBMD_OBS_ENERGY = 1u,    /* kinetic, potential, temperature, conserved quantity     */
    BBMD_OBS_VIRIAL = 2u,    /* virial W = sum_{i<j} r_ij . F_ij and pressure            */
    BBMD_OBS_MOMENTUM = 4u,  /* total momentum                                          */
    BBMD_OBS_GR = 8u,        /* partial g_ab(r) (Sec. 4)                                */
    BBMD_OBS_MSD = 16u,      /* mean-square displacement per species since SET_REF      */
    BBMD_OBS_FS = 32u,       /* self-intermediate scattering F_s(k, t) since SET_REF    */
    BBMD_OBS_SET_REF = 64u   /* store the current unwrapped positions as the reference
                                of the time origin args->origin (before MSD / FS)       */
};

/* Time origins of MSD and F_s: SET_REF stores the unwrapped positions as reference
 * `origin`, MSD / FS measure against reference `origin` (each origin holds 3n doubles of
 * device memory once set), so averages over several time origins need no host copies. */
#define BBMD_MAX_ORIGINS 16

typedef struct {
    int32_t nbins;   /* g(r) bins (0 = 500)  */
    double rmax;     /* g(r) range (0 = 5.0) */
    double k;        /* F_s wave number (0 = 7.25) */
    int32_t origin;  /* time origin of SET_REF / MSD / FS, in [0, BBMD_MAX_ORIGINS) */
} bbmd_obs_args;

/* Results of bbmd_observe.  gr_counts[(a*2+b)*nbins + q] counts ordered pairs (i in a,
 * j in b, j != i) with floor(r/dr) = q, dr = rmax/nbins, r from the exact r^2 rule;
 * gr[...] = V n_ab / (N_a N'_b (4 pi/3)(r_{q+1}^3 - r_q^3)), N'_b = N_b - (a == b).
 * Both pointers are caller-owned (4*nbins entries) and may be NULL. */
typedef struct {
    double ke, pe, virial, pressure, temperature;
    double momentum[3];
    double xi, eta, conserved;  /* NH variables; conserved = K + U + Q xi^2/2 + g T eta   */
    int64_t step;               /* steps taken since creation                           */
    int64_t n_rebuilds;         /* list / cell rebuilds since creation                  */
    uint64_t* gr_counts;
    double* gr;
    double msd[2];
    double fs[2];
} bbmd_obs;

/* Static facts of a handle. */
typedef struct {
    int64_t n;
    int32_t fix_exponent;    /* k of the position unit 2^-k                */
    int32_t nc[3];           /* cells per axis                             */
    int64_t cell_side_fix[3];/* D per axis in units of 2^-k                */
    int32_t list_capacity;
    int32_t stencil_capacity;
    int64_t device_bytes;    /* device memory held by the handle           */
    int32_t block_z;         /* block shape code in use (see bbmd_params)  */
    float shape_force_ms[4]; /* autotuner: force / list-build ms per launch   */
    float shape_list_ms[4];  /*   for block_z = 1, 2, 4, 8, measured on a     */
                             /*   part of the box and scaled to all of it     */
                             /*   (0 = not timed)                             */
} bbmd_info;

/* Create a system of n particles in a periodic box (Sec. 2).
 * box[3]: sides (>= 1).  species: n labels (host, required).
 * pos: n x 3 host positions, or NULL for the FCC lattice of 4 m^3 sites (n must equal
 *   4 m^3) with site i = 4 (ix + m (iy + m iz)) + b at ((ix,iy,iz) + basis_b + 1/4) L/m.
 * vel: n x 3 host velocities, or NULL for Maxwell-Boltzmann velocities at T0 drawn from
 *   the counter-based SplitMix64/Box-Muller generator under seed (net momentum removed,
 *   then scaled to 2K/(3n-3) = T0).
 * stream: a cudaStream_t, or NULL for a non-blocking stream created and owned by the
 *   handle (the legacy default stream cannot hold the captured step graph).
 * alloc: NULL = cudaMalloc.
 * On success *out receives the handle, the first list is built and the forces of the
 * initial positions are computed. */
/* Non-finite input positions or velocities and species labels other than 0 and 1 are
 * rejected with BBMD_ERR_ARG, before any device work. */
bbmd_status bbmd_create(const bbmd_params* params, int64_t n, const double box[3],
                        const uint8_t* species, const double* pos, const double* vel,
                        double T0, uint64_t seed, void* stream, const bbmd_alloc* alloc,
                        bbmd_sim** out);

/* Release all device memory of the handle (NULL is ignored). */
void bbmd_destroy(bbmd_sim* sim);

/* Advance nsteps velocity-Verlet steps of size dt (Sec. 2.3.2) under the thermostat
 * (NULL = NVE).  Asynchronous: returns after enqueueing on the handle's stream.  The list
 * is rebuilt on the device when needed, without a host round trip.
 * The last step's closing half kick (and Nose-Hoover scale) is left pending in the stored
 * velocities: the next call with the same dt applies it within its first velocity update,
 * as two steps of one call do (so split calls give the trajectory of one call, bit for
 * bit); a call with another dt, bbmd_get_state, bbmd_set_state, bbmd_minimize, bbmd_tune
 * and bbmd_rebuild apply it first; bbmd_observe reports the finished velocities' kinetic
 * energy and momentum without storing them. */
bbmd_status bbmd_step(bbmd_sim* sim, int64_t nsteps, double dt, const bbmd_thermostat* thermo);

/* Phases timed by bbmd_step_profiled. */
enum {
    BBMD_PHASE_INTEGRATE = 0,   /* kick + drift + wrap + frame copy + rebuild trigger          */
    BBMD_PHASE_REBUILD = 1,     /* binning, scan, scatter, per-cell order, reorder (gated)     */
    BBMD_PHASE_LIST = 2,        /* Verlet list build (gated)                                   */
    BBMD_PHASE_FORCE = 3,       /* pair forces (+ kinetic-energy partials when thermostatted)  */
    BBMD_PHASE_FINALIZE = 4,    /* reduction and thermostat update                             */
    BBMD_PHASE_COUNT = 5
};

/* Same computation as bbmd_step, with every phase launched on its own and bracketed by CUDA
 * events on the handle's stream; ms[BBMD_PHASE_COUNT] receives the summed device time of
 * each phase over the nsteps steps and *rebuilds the number of rebuilds that ran (either
 * may be NULL).  Synchronising.  Used to attribute step time to kernels. */
bbmd_status bbmd_step_profiled(bbmd_sim* sim, int64_t nsteps, double dt,
                               const bbmd_thermostat* thermo, double* ms, int64_t* rebuilds);

/* Measure the observables selected by mask at the current state (synchronising).  args may
 * be NULL for the defaults (time origin 0).  out->gr_counts / out->gr are filled when
 * non-NULL and GR is set.  MSD / FS of an origin never set by SET_REF -> BBMD_ERR_STATE.
 * ENERGY / VIRIAL evaluate pair energies in FP64 from the exact integer positions in
 * mixed precision too (the forces of the step stay the FP32 kernel's). */
bbmd_status bbmd_observe(bbmd_sim* sim, uint32_t mask, const bbmd_obs_args* args,
                         bbmd_obs* out);

/* Steepest descent x += h F, h = min(hmax, dmax / max_i |F_i|), nsteps times; the forces
 * of the final positions are left valid.  Velocities are untouched. */
bbmd_status bbmd_minimize(bbmd_sim* sim, int64_t nsteps, double hmax, double dmax);

/* Copy the state to host arrays in id order (each may be NULL): positions wrapped into
 * [0, L) (n x 3), velocities (n x 3), image counters (n x 3, box crossings since creation).
 * Synchronising. */
bbmd_status bbmd_get_state(bbmd_sim* sim, double* pos, double* vel, int32_t* image);

/* Replace positions (n x 3, quantised as in bbmd_create), velocities (n x 3) and image
 * counters (n x 3, NULL = zeros) from host arrays in id order.  Species are kept.  The
 * list is rebuilt and forces recomputed; the thermostat variables are kept.  Non-finite
 * positions or velocities (checked on the device after the upload, before anything of the
 * state is replaced) return BBMD_ERR_ARG with the state unchanged.  Synchronising. */
bbmd_status bbmd_set_state(bbmd_sim* sim, const double* pos, const double* vel,
                           const int32_t* image);

/* Forces of the current positions (n x 3, id order) and, when u is non-NULL, per-particle
 * potential energy (half of each pair energy).  Recomputes on the device; synchronising. */
bbmd_status bbmd_get_forces(bbmd_sim* sim, double* F, double* u);

/* Forces (m x 3) and, when u is non-NULL, per-particle energies (m) of the particles ids[0..m)
 * at the current positions (recomputed on the device as in bbmd_get_forces); copies only
 * the m results to the host, for sampling large systems.  Synchronising. */
bbmd_status bbmd_get_forces_ids(bbmd_sim* sim, const int64_t* ids, int64_t m, double* F,
                                double* u);

/* Cell of each particle at the last rebuild (n entries, id order):
 * (az * ncy + ay) * ncx + ax.  Synchronising. */
bbmd_status bbmd_get_cells(bbmd_sim* sim, int64_t* cell);

/* Current Verlet list as sets of ids.  ids: the m particle ids to report (NULL = all n,
 * in id order).  offsets[m+1] (or [n+1]) receives the prefix of the list lengths and, when
 * nbr is non-NULL, nbr[offsets[s] .. offsets[s+1]) the ascending ids of the list of the
 * s-th requested particle (cap entries available; BBMD_ERR_ARG if too small).  Verlet mode
 * only (BBMD_ERR_STATE otherwise).  Synchronising. */
bbmd_status bbmd_get_neighbors(bbmd_sim* sim, const int64_t* ids, int64_t m, int64_t* offsets,
                               int64_t* nbr, int64_t cap);

/* Re-run the block-shape autotuner of bbmd_create on the current state (creation times the
 * shapes on the initial state, e.g. a lattice; a liquid can favour another shape), rebuild
 * the lists for the shape chosen and recompute the forces.  The list build is weighted by
 * the rebuilds per step observed since the previous tuning (creation weighs it 1/4).
 * Nothing changes when params.block_z fixed the shape.  Synchronising. */
bbmd_status bbmd_tune(bbmd_sim* sim);

/* Force a rebuild (binning, reorder and list) at the current positions. */
bbmd_status bbmd_rebuild(bbmd_sim* sim);

bbmd_status bbmd_get_info(const bbmd_sim* sim, bbmd_info* info);

/* ---- Replica batches --------------------------------------------------------------
 * Many independent systems ("replicas": e.g. one mixture per temperature, of uneven sizes)
 * advanced together.  Each replica is a complete handle with its own box, particles,
 * cells, lists and thermostat variables; bbmd_step_batch advances all of them with one
 * persistent kernel launch for up to 1024 steps (bbmd_batch_set_mode) or one CUDA graph
 * launch per step: groups of replicas on parallel branches of that graph, one kernel
 * launch per phase covering every replica of a group.  The paper runs one system at a time (Sec. 3, 4); a batch fills the GPU with
 * systems far smaller than it. */
typedef struct bbmd_batch bbmd_batch;

/* Create n_rep >= 1 replicas sharing params (and one block shape: params.block_z, 0 for
 * 2 x 2 x 4).  Replica r: n[r] particles in the box
 * box[3r .. 3r+2]; species[r] (host, n[r] labels, required); positions pos[r] and
 * velocities vel[r] as in bbmd_create (pos or vel NULL, or an entry NULL, for the
 * device-generated FCC lattice / Maxwell-Boltzmann velocities at T0[r] under seed + r).
 * stream: a cudaStream_t shared by all replicas, or NULL for one owned by the batch.
 * alloc: as bbmd_create.  On failure nothing stays allocated and *out is NULL. */
bbmd_status bbmd_create_batch(const bbmd_params* params, int32_t n_rep, const int64_t* n,
                              const double* box, const uint8_t* const* species,
                              const double* const* pos, const double* const* vel,
                              const double* T0, uint64_t seed, void* stream,
                              const bbmd_alloc* alloc, bbmd_batch** out);

/* Advance every replica by nsteps steps of size dt (Sec. 2.3.2).  thermo: n_rep
 * thermostats, thermo[r] for replica r, all of the same kind; NULL = NVE for all.
 * Asynchronous, like bbmd_step. */
bbmd_status bbmd_step_batch(bbmd_batch* b, int64_t nsteps, double dt,
                            const bbmd_thermostat* thermo);

/* Handle of replica r, owned by the batch and valid until bbmd_destroy_batch; every
 * single-system call (observe, get/set state, minimize, step, ...) works on it.  NULL if r
 * is out of range. */
bbmd_sim* bbmd_batch_replica(bbmd_batch* b, int32_t r);

int32_t bbmd_batch_size(const bbmd_batch* b);

/* Branches of the batch step graph (default 8): the replicas are split into this many
 * groups of about equal particle count; within a group one launch per phase covers every
 * replica, and the groups run concurrently.  Takes effect at the next bbmd_step_batch. */
bbmd_status bbmd_batch_set_branches(bbmd_batch* b, int32_t branches);

/* Step path of a batch.  AUTO (the default): the persistent step when it applies, else the
 * graph.  PERSISTENT: one cooperative kernel launch runs up to 1024 whole steps of every
 * replica.  Each phase of a replica's step (integrate, rebuild trigger, the gated sort
 * chain and list build, forces, finalize) is cut into work items with the CTA index and
 * count of the per-replica kernels, so the states are bit for bit those of stepping each
 * replica alone.  All resident CTAs take the items from one queue, step after step and
 * phase after phase; an item starts once its replica's previous phase has finished, so
 * the phases and steps of different replicas overlap.  It applies to mixed precision with
 * block shape 2 x 2 x 4 (the batch default) on a device with cooperative launch;
 * otherwise bbmd_step_batch returns BBMD_ERR_STATE.  A wait gives up after a second
 * (bbmd_batch_set_wait_limit); the replicas then report BBMD_ERR_TIMEOUT at their next
 * synchronising call.  GRAPH: one CUDA graph launch per step (bbmd_batch_set_branches). */
enum { BBMD_BATCH_AUTO = 0, BBMD_BATCH_GRAPH = 1, BBMD_BATCH_PERSISTENT = 2 };
bbmd_status bbmd_batch_set_mode(bbmd_batch* b, int32_t mode);

/* Limit of each dependency wait of the persistent step, in ns (default 1e9; ns >= 1, else
 * BBMD_ERR_ARG).  A wait that runs out raises an abort flag: every CTA of the launch
 * returns at its next work item, the rest of the call's launches return at once, and
 * every replica reports BBMD_ERR_TIMEOUT at its next synchronising call.  The replicas'
 * states are then those of partly completed steps (destroy the batch); the device context
 * stays usable.  The paper has no counterpart (failure detection of this design). */
bbmd_status bbmd_batch_set_wait_limit(bbmd_batch* b, uint64_t ns);

/* 1 if the next bbmd_step_batch takes the persistent step, else 0. */
int32_t bbmd_batch_uses_persistent(const bbmd_batch* b);

/* Release every replica and the batch (NULL is ignored). */
void bbmd_destroy_batch(bbmd_batch* b);

/* Message of the last failed batch call ("" if none). */
const char* bbmd_batch_last_error(const bbmd_batch* b);

/* Fixed size of the device scratch used by bbmd_gr_counts_noalloc (int32 entries, 16 MiB)
 * and its largest bin count. */
#define BBMD_NOALLOC_GR_SCRATCH_INTS (1 << 22)
#define BBMD_NOALLOC_GR_MAX_BINS 4096

/* The g(r) pair counts of bbmd_observe(BBMD_OBS_GR) (same definition, same layout as
 * bbmd_obs.gr_counts: counts[(a*2+b)*nbins + q], 4*nbins entries, caller-owned host array)
 * computed without allocating any device memory.  The paper has no counterpart: it is a
 * library variant of the g(r) observable for callers that must not allocate.
 *   nbins <= 0 -> 500, rmax <= 0 -> 5.0 (as bbmd_observe); nbins <= 4096.
 *   Scratch: one fixed device array inside the library, BBMD_NOALLOC_GR_SCRATCH_INTS int32
 *   entries plus 4*4096 counters.  When the box holds at least 3 cells of side rmax per
 *   axis, the coarse-grid search needs 2n + 3(ncg + 1) entries (ncg = number of those
 *   cells); a larger need is rejected with BBMD_ERR_ARG before anything is launched (use
 *   bbmd_observe then).  Smaller boxes take the all-pairs path, which needs no int32
 *   scratch.
 *   Nothing has to start at zero: each call clears the counters and the coarse-cell counts
 *   it uses before filling them.
 *   The first call on a device looks up the array's address (cudaGetSymbolAddress); make
 *   that first call before any stream capture on the device.
 *   Calls that overlap in time on one device, from any handles or threads, share the one
 *   array and race: serialise them.
 * Synchronising. */
bbmd_status bbmd_gr_counts_noalloc(bbmd_sim* sim, int32_t nbins, double rmax, uint64_t* counts);

/* Message of the last failed call on this handle ("" if none). */
const char* bbmd_last_error(const bbmd_sim* sim);

/* Measured peak fused multiply-add rate of the current device, in TFLOP/s (2 flops per
 * FMA): precision BBMD_PREC_MIXED -> FP32, BBMD_PREC_FP64 -> FP64.  *sm_count (may be
 * NULL) receives the device's multiprocessor count.  A measurement helper: the roofline
 * denominator of the pair-force kernels, which are bound by arithmetic issue, not by
 * memory; the paper has no counterpart.  Every thread of 8 CTAs of 256 threads per SM
 * runs 8 independent FMA chains with no memory traffic; the best of 3 timed launches
 * (CUDA events) after a warm-up launch is reported.  Allocates a few KB of device memory
 * for the duration of the call; synchronising; about half a second. */
bbmd_status bbmd_fma_peak(int32_t precision, int32_t* sm_count, double* tflops);

/* Measured rate of shared-memory scatter-adds on the current device, in adds per second
 * over the whole GPU: kind 0 = 64-bit integer adds of a float converted to 2^32 fixed
 * point (the deterministic reaction update of a half-list force kernel), 1 = 32-bit
 * integer adds, 2 = FP32 adds.  Each thread of 4 CTAs of 256 threads per SM adds at
 * addresses that differ across a warp's lanes (no bank conflicts: the most favourable
 * case); best of 3 timed launches after a warm-up.  A measurement helper behind the
 * choice of a full Verlet list; the paper has no counterpart.  Allocates a few bytes of
 * device memory for the duration of the call; synchronising. */
bbmd_status bbmd_smem_scatter_rate(int32_t kind, double* adds_per_s);

#ifdef __cplusplus
}
#endif
#endif
