// Internal definitions shared by the CUDA translation units of libbbmd (not installed).
//
// Data layout in device memory (sorted order = by (cell, id) after each rebuild):
//   x[3][npad]   int64   positions in units of 2^-k (SoA per axis)
//   v[3][npad]   int64   velocities in units of 2^-52
//   img[3][npad] int32   box crossings
//   id[npad]     int32   particle id;  sp[npad] uint8 species
//   rel[npad]    float4  position relative to the frame of its build cell, w = species (0.f / 1.f)
//   relb[npad]   float4  the same at the last rebuild, w = (cell << 1) | species
//   F[npad]      float4  mixed-precision force (w = per-particle energy on energy passes)
//   Fd[3][npad]  double  FP64-form force
//   list[lcap8][npad][8] uint16  Verlet list: offsets into the staged region (the cells
//                                 around the particle's block of cells)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bbmd.h"

namespace bbmd {

constexpr int kVelExp = 52;            // velocity unit 2^-52
// Block shapes of the force / list kernels, by code bz: 1, 2 and 4 are blocks of 2 x 2 x bz
// cells, 8 is a block of 4 x 4 x 2 cells (32 cells, like 2 x 2 x 8, but its cells are at
// most 2 cells from the block's middle along every axis).  One CTA works on a block at a
// time, with the (X + 2) x (Y + 2) x (Z + 2) cells around it staged in shared memory.
// k_force.cu is compiled once per shape (namespace z<bz>); a handle runs the shape chosen
// at creation.
constexpr int kShapes[4] = {1, 2, 4, 8};
__host__ __device__ constexpr int block_xy_of(int bz) { return bz == 8 ? 4 : 2; }
__host__ __device__ constexpr int block_zc_of(int bz) { return bz == 8 ? 2 : bz; }
__host__ __device__ constexpr int block_cells_of(int bz) {
    return block_xy_of(bz) * block_xy_of(bz) * block_zc_of(bz);
}
__host__ __device__ constexpr int region_cells_of(int bz) {
    return (block_xy_of(bz) + 2) * (block_xy_of(bz) + 2) * (block_zc_of(bz) + 2);
}
constexpr int kMaxPartials = 8192;     // per-block FP64 partial sums
constexpr float kBand = 1e-5f;         // relative band around a threshold for the FP64 re-test

// status bits (sticky, OR-ed on the device)
enum : int32_t {
    ST_LIST_OVERFLOW = 1,
    ST_STENCIL_OVERFLOW = 2,
    ST_NONFINITE = 4,
    ST_VEL_RANGE = 8,
    ST_TIMEOUT = 16,
};

struct DevScalars {
    double xi, eta;          // Nose-Hoover friction and its time integral
    double K;                // kinetic energy of the stored (full-step) velocities
    double s_next;           // velocity scale applied by the next integrate kernel
    double s_end;            // scale applied by the finish kernel
    double dt, T_start, T_end, tau, g;
    float hdt[2];            // dt / (2 m_a) in FP32 (set with dt)
    double T_last;           // target temperature of the last step
    double pe, w;            // last energy pass
    double kin_last;         // K of the last finalize (before NH scaling)
    double maxf;             // steepest descent: max |F|
    long long step, n_rebuilds;
    int step_in_call, n_in_call, kind;
    int pending;             // 1: the last step's closing half kick (scaled by s_end) is not
                             //    yet in the stored velocities (applied by the next call's
                             //    first update, or by the finish kernel)
    int rebuild;             // 1: the gated rebuild kernels run in this step
    int near;                // 1: some displacement of this step exceeds half the threshold
    int status;              // ST_* bits
    int bad_input;           // set_state: 1 if an uploaded value is not finite
    int list_short;          // 1: the stored lists were cut at the capacity; the forces come
                             //    from the cell stencil until the lists are rebuilt larger
    int max_len;             // longest cut list of the last build (entries)
};

struct PairTab {
    // FP32 tables [a*2+b]
    float rc2lo[4], rc2hi[4];     // rcut^2 (1 -/+ band)
    float R2lo[4], R2hi[4];       // (rcut + skin)^2 (1 -/+ band)
    float sig2[4], sig2lo[4], eps48[4], eps4[4], vshift[4], fcut[4], frc[4];
    // FP64 tables: exact decisions and the FP64 form
    double rc2[4], R2[4], dsig2[4], deps48[4], deps4[4], dvshift[4], dfcut[4], drc[4];
    long long rcfix[4];           // ceil(rcut * 2^k): |dx| beyond it on some axis -> no pair
    float mass[2];
    double dmass[2];
    int potential, shift;
};

struct alignas(16) DevSim {
    int64_t n, npad;
    int32_t ncell, nc[3];
    int64_t D[3], Lfix[3];
    int32_t kexp;
    float sx;                // 2^-k
    double sxd;
    int32_t lcap8, smax;     // list capacity / 8; staged capacity of one block region
    int32_t block_z;         // block shape code (one of kShapes; block_xy_of, block_zc_of)
    int32_t region_cells;    // cells staged per block: 4 x 4 x (block_z + 2)
    int64_t nblocks;         // blocks of the shape (block_xy_of x block_xy_of x block_zc_of)
    float halfL[3];          // L/2 (FP32) per axis
    int32_t nbr_mode, precision;
    float disp2;             // steepest descent: rebuild threshold on |x - x_build|^2
    float disp_thr;          // rebuild when two particles of the same or neighbouring build
                             // cells moved beyond it together (skin, FP32, conservative)
    float disp_far;          // rebuild when any two particles moved beyond it together
                             // (D_min - rc_max: pairs whose build cells are two apart)
    float* disp;             // [npad] displacement since the last build (integrate)
    float2* mtop;            // [ncell] two largest displacements per build cell
    PairTab pt;
    uint64_t* x; int64_t* v; int32_t* img; int32_t* id; uint8_t* sp;
    uint64_t* x2; int64_t* v2; int32_t* img2; int32_t* id2; uint8_t* sp2;
    float4 *rel, *relb, *F;
    double* Fd;
    double* ud;              // per-particle FP64 energy (energy passes)
    int32_t *key, *cell_start, *count, *cursor, *perm, *perm_tmp, *scan_part;
    uint16_t* list;
    uint16_t* rows;          // per particle: rows (8 entries each) of its Verlet list
    double* partials;        // [kMaxPartials][4]
    DevScalars* sc;
    int32_t grid_part;       // grid of per-particle grid-stride kernels
    int32_t grid_cell;       // grid of the force kernel (kBlockWarps warps per CTA)
    int32_t grid_list;       // grid of the list-build kernel
};

// ---------------------------------------------------------------- conversions ----

// Correctly rounded int64 -> float using 32-bit operations (no FP64 pipe).
__device__ __forceinline__ float i64_to_f32(long long v) {
    if (v == 0) return 0.0f;
    unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
    int lz = __clzll(a);
    unsigned long long m = a << lz;                    // MSB at bit 63
    unsigned int hi = (unsigned int)(m >> 32);
    unsigned int lo = (unsigned int)m;
    hi |= (lo != 0u);                                  // sticky bit keeps rounding exact
    float f = __uint2float_rn(hi);                     // 32 -> 24 bits, round to nearest
    // multiply by 2^(32 - lz) exactly (power of two built from its bit pattern)
    int e = 127 + 32 - lz;
    f *= __int_as_float(e << 23);
    return v < 0 ? -f : f;
}

// Approximate int64 -> float (error about one ulp), for velocities.
__device__ __forceinline__ float i64_to_f32_fast(long long v) {
    int hi = (int)(v >> 32);
    unsigned int lo = (unsigned int)v;
    return fmaf((float)hi, 4294967296.0f, __uint2float_rn(lo));
}

// float (already scaled, |y| < 2^62) -> int64 rounded to nearest, using 32-bit converts.
__device__ __forceinline__ long long f32_to_i64(float y) {
    float hf = floorf(y * 2.3283064365386963e-10f);    // y / 2^32 (exact), floored
    float lf = fmaf(-hf, 4294967296.0f, y);            // exact low part in [0, 2^32)
    long long hi = (long long)__float2int_rn(hf);
    unsigned long long lo = (unsigned long long)__float2uint_rn(lf);
    return (long long)(((unsigned long long)hi << 32) + lo);
}

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// ------------------------------------------------------------ cells and frames ----

// Cell index along one axis: a = min(nc-1, x / D) by a float estimate and exact fix-up.
__device__ __forceinline__ int cell_axis(long long x, long long D, int nc) {
    float est = __fdividef(i64_to_f32_fast(x), i64_to_f32_fast(D));
    int a = (int)est;
    if (a < 0) a = 0;
    if (a > nc - 1) a = nc - 1;
    while (a > 0 && (long long)a * D > x) --a;
    while (a < nc - 1 && (long long)(a + 1) * D <= x) ++a;
    return a;
}

// Frame point of cell a along one axis (the cell's centre on the D grid).
__device__ __forceinline__ long long frame_axis(int a, long long D) {
    return (long long)a * D + (D >> 1);
}

// Minimum-image reduction of an integer displacement |d| < 3L/2: d > L/2 -> d - L,
// d < -L/2 -> d + L.  For integer d the tests d > floor(L/2) and d < -floor(L/2) are the
// same decisions as 2d > L and 2d < -L, without the overflow of 2d when L is near 2^62.
__device__ __forceinline__ long long min_image(long long d, long long L) {
    const long long h = L >> 1;
    if (d > h) d -= L;
    else if (d < -h) d += L;
    return d;
}

__device__ __forceinline__ void cell_coords(int c, const int32_t* nc, int& ax, int& ay, int& az) {
    ax = c % nc[0];
    int t = c / nc[0];
    ay = t % nc[1];
    az = t / nc[1];
}

// Exact r^2 rule in FP64 (the same IEEE operations the oracle performs).
__device__ __forceinline__ double r2_exact(const DevSim& s, int64_t i, int64_t j) {
    double d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        long long dx = (long long)s.x[a * s.npad + j] - (long long)s.x[a * s.npad + i];
        dx = min_image(dx, s.Lfix[a]);
        d[a] = __dmul_rn(__ll2double_rn(dx), s.sxd);
    }
    return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
}

__device__ __forceinline__ void set_status(const DevSim& s, int bits) {
    atomicOr(&s.sc->status, bits);
}

// ------------------------------------------------------------------ replica batches ----
// A batch launch runs one phase for every replica of a batch: replica r owns the CTAs
// first[r] .. first[r + 1] - 1 of the grid.  Each kernel of the step is written once as a
// body taking (system, CTA index within it, CTA count of it) and wrapped twice: for one
// system (DevSim by value, blockIdx / gridDim) and for a batch (the replica's DevSim copied
// to shared memory).
struct ManySims {
    const DevSim* sims;     // nrep systems (device memory)
    const int32_t* first;   // nrep + 1 CTA offsets (device memory)
    int32_t nrep;
};

// The replica of this CTA: copies its DevSim into sh and returns the CTA's index and count
// within the replica.  Every thread of the CTA calls it once, first (it synchronises).
__device__ __forceinline__ void load_replica(const ManySims& m, DevSim& sh, int& lb, int& lg) {
    __shared__ int rep_of_cta;
    if (threadIdx.x == 0) {
        int lo = 0, hi = m.nrep - 1;  // the last replica whose first CTA is <= blockIdx.x
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (m.first[mid] <= (int)blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        rep_of_cta = lo;
    }
    __syncthreads();
    const int r = rep_of_cta;
    const int4* src = reinterpret_cast<const int4*>(m.sims + r);
    int4* dst = reinterpret_cast<int4*>(&sh);
    for (int k = threadIdx.x; k < (int)(sizeof(DevSim) / 16); k += blockDim.x) dst[k] = src[k];
    lb = (int)blockIdx.x - m.first[r];
    lg = m.first[r + 1] - m.first[r];
    __syncthreads();
}

#define BBMD_ONE_AND_MANY(bounds, name, body)                                             \
    __global__ void __launch_bounds__(bounds) name(DevSim s) {                            \
        body(s, (int)blockIdx.x, (int)gridDim.x);                                         \
    }                                                                                     \
    __global__ void __launch_bounds__(bounds) name##_many(ManySims m) {                   \
        __shared__ DevSim sh;                                                             \
        int lb, lg;                                                                       \
        load_replica(m, sh, lb, lg);                                                      \
        body(sh, lb, lg);                                                                 \
    }

// ------------------------------------------------------------ launch wrappers ----
// (defined in the .cu files; all enqueue on `st`)

// sort / rebuild chain (gated on sc->rebuild unless noted)
void launch_rebuild_chain(const DevSim& s, cudaStream_t st);
// Per block shape (namespace z1, z2, z4, z8; defined in k_force.cu compiled per shape):
//   prepare_force_kernels  one-time kernel attributes (call before any stream capture)
//   force/list_blocks_per_sm  resident CTAs per SM for this handle's shared memory
//   launch_force   forces; energy: also per-particle energy and virial partials; ke: NH
//                  kinetic partials
//   launch_list_build  Verlet list build (gated)
#define BBMD_SHAPE_API(ns)                                                             \
    namespace ns {                                                                     \
    bool prepare_force_kernels();                                                      \
    void launch_force_many(const ManySims& m, int total, bool fp64, bool cell, bool ke,    \
                           bool fshift, int smax_max, cudaStream_t st);                \
    void launch_list_build_many(const ManySims& m, int total, int smax_max,             \
                                cudaStream_t st);                                      \
    int force_blocks_per_sm(const DevSim& s);                                          \
    int list_blocks_per_sm(const DevSim& s);                                           \
    int block_threads();                                                               \
    void launch_force(const DevSim& s, cudaStream_t st, bool energy, bool ke);         \
    void launch_list_build(const DevSim& s, cudaStream_t st);                          \
    }
BBMD_SHAPE_API(z1)
BBMD_SHAPE_API(z2)
BBMD_SHAPE_API(z4)
BBMD_SHAPE_API(z8)
#undef BBMD_SHAPE_API

// Block shape of the persistent batch step (k_force.cu compiled for it holds the kernel).
#ifndef BBMD_PERSIST_Z
#define BBMD_PERSIST_Z 4
#endif
constexpr int kPersistZ = BBMD_PERSIST_Z;
// Persistent batch step (block shape 2 x 2 x kPersistZ, mixed precision): one cooperative launch
// runs every phase of many steps for every replica.  Work items (phase, replica, CTA
// index, CTA count) come from one queue, step-major and phase-major within a step; an
// item starts once its replica's previous non-empty phase has finished.
enum {
    kPhIntegrate = 0, kPhCelltop, kPhCheck, kPhZero, kPhBin, kPhScan, kPhScatter, kPhCellsort,
    kPhGather, kPhCopyback, kPhList, kPhForce, kPhFinalize, kPhases
};
struct PersistentStep {
    const DevSim* sims;       // nrep replica systems (device copies)
    const int4* items;        // nitems work items {phase, replica, lb, lg}, phase-major
    const int32_t* need;      // [nrep][kPhases] items per replica and phase
    const int32_t* dep;       // [nrep][kPhases] the phase an item waits for (-1: none)
    int32_t* done;            // [nrep][kPhases] finished items, zero at launch
    uint32_t* head;           // queue head, zero at launch
    int32_t* abort;           // raised when a wait gives up (stays raised for the call)
    int32_t nrep, nitems;     // replicas; work items of one step
    int32_t nsteps;           // steps of this launch (items nitems * nsteps)
    uint64_t wait_ns;         // a dependency wait gives up after this many ns
};
#define BBMD_PERSIST_NS2(n) z##n
#define BBMD_PERSIST_NS1(n) BBMD_PERSIST_NS2(n)
#define BBMD_PERSIST_NS BBMD_PERSIST_NS1(BBMD_PERSIST_Z)
namespace BBMD_PERSIST_NS {
bool prepare_persistent();                    // kernel attributes (before any capture)
int persistent_blocks_per_sm(int smax_max);   // resident CTAs per SM
cudaError_t launch_persistent_step(const PersistentStep& a, int grid, int smax_max, bool ke,
                                   bool fshift, cudaStream_t st);
}  // namespace

#define BBMD_SHAPE_DISPATCH(bz, call)          \
    switch (bz) {                              \
        case 1: return z1::call;               \
        case 2: return z2::call;               \
        case 4: return z4::call;               \
        default: return z8::call;              \
    }
inline bool prepare_force_kernels() {
    return z1::prepare_force_kernels() && z2::prepare_force_kernels() &&
           z4::prepare_force_kernels() && z8::prepare_force_kernels();
}
inline int force_blocks_per_sm(const DevSim& s) { BBMD_SHAPE_DISPATCH(s.block_z, force_blocks_per_sm(s)) }
inline int list_blocks_per_sm(const DevSim& s) { BBMD_SHAPE_DISPATCH(s.block_z, list_blocks_per_sm(s)) }
inline void launch_force(const DevSim& s, cudaStream_t st, bool energy, bool ke) {
    BBMD_SHAPE_DISPATCH(s.block_z, launch_force(s, st, energy, ke))
}
inline void launch_list_build(const DevSim& s, cudaStream_t st) {
    BBMD_SHAPE_DISPATCH(s.block_z, launch_list_build(s, st))
}
#undef BBMD_SHAPE_DISPATCH
// batch launches: one launch runs the phase for every replica of m; first[] of m must
// hold each replica's CTA count of that phase (grid_part for the per-particle kernels,
// the scan grid, 1 for the per-replica reductions)
int scan_grid(const DevSim& s);
void launch_rebuild_chain_many(const ManySims& part, const ManySims& scan, const ManySims& one,
                               int total_part, int total_scan, int nrep, cudaStream_t st);
void launch_integrate_many(const ManySims& part, int total, bool fp64, cudaStream_t st);
// rebuild trigger from the per-cell displacements of this step (after integrate)
void launch_check(const DevSim& s, cudaStream_t st);
void launch_check_many(const ManySims& part, int total, cudaStream_t st);
void launch_finalize_many(const ManySims& one, int nrep, bool ke, cudaStream_t st);
// integrator pieces
void launch_begin(const DevSim& s, cudaStream_t st, int64_t nsteps, double dt,
                  const bbmd_thermostat* th);
void launch_integrate(const DevSim& s, cudaStream_t st);
void launch_finalize(const DevSim& s, cudaStream_t st, bool ke);
// apply the closing half kick and NH scale a call left pending (no-op when none is)
void launch_finish(const DevSim& s, cudaStream_t st);
void launch_state_sums(const DevSim& s, cudaStream_t st);          // KE, P partials -> sc->K etc.
void launch_reduce_partials(const DevSim& s, cudaStream_t st, int nq, double* out_dev);
void launch_init_fcc(const DevSim& s, cudaStream_t st, int m, double jitter, uint64_t seed);
void launch_init_mb(const DevSim& s, cudaStream_t st, double T0, uint64_t seed, double* tmp3);
void launch_sd_step(const DevSim& s, cudaStream_t st, double hmax, double dmax);
void launch_clear_rebuild(const DevSim& s, cudaStream_t st);
// unwrapped positions by id (3 x n doubles) into ref / MSD and F_s against ref
void launch_set_ref(const DevSim& s, cudaStream_t st, double* ref);
void launch_msd_fs(const DevSim& s, cudaStream_t st, const double* ref, double kvec,
                   double* out_dev);
int launch_gr(const DevSim& s, cudaStream_t st, int nbins, double rmax,
              unsigned long long* counts_dev, int32_t* scratch_i32, float4* scratch_f4,
              int64_t scratch_n);
void launch_unpack_state(const DevSim& s, cudaStream_t st, double* pos, double* vel,
                         int32_t* img);   // device buffers, id order
void launch_pack_state(const DevSim& s, cudaStream_t st, const double* pos, const double* vel,
                       const int32_t* img, bool species_from_current);
void launch_unpack_forces(const DevSim& s, cudaStream_t st, double* F, double* u);
// sc->bad_input = 1 if one of the m doubles at a (device) is not finite
void launch_check_finite(const DevSim& s, cudaStream_t st, const double* a, int64_t m);
void launch_unpack_cells(const DevSim& s, cudaStream_t st, int64_t* cell);
void launch_forces_of_ids(const DevSim& s, cudaStream_t st, const int32_t* slot_of,
                          const int64_t* ids, int64_t m, double* F, double* u);
// Neighbour lists by id.  sel: slots of the m requested particles (NULL = all, output
// in id order).
void launch_slot_of(const DevSim& s, cudaStream_t st, int32_t* slot_of);
void launch_list_counts(const DevSim& s, cudaStream_t st, const int32_t* sel, int64_t m,
                        int64_t* counts);
void launch_list_ids(const DevSim& s, cudaStream_t st, const int32_t* sel, int64_t m,
                     const int64_t* offsets, int64_t* nbr);

}  // namespace bbmd
