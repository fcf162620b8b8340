// C ABI of libbbmd (declared in include/bbmd.h): handle life cycle, device memory plan,
// the captured per-step CUDA graph and the synchronising queries.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "bbmd_internal.cuh"

using namespace bbmd;

struct bbmd_sim {
    bbmd_params P;
    DevSim d;
    double box[3];
    cudaStream_t st = nullptr;
    bool own_stream = false;
    bbmd_alloc alloc;
    bool have_alloc = false;
    std::vector<std::pair<void*, size_t>> blocks;
    int64_t bytes = 0;
    std::string err;
    double* dout = nullptr;          // device scratch for reduction results (64 doubles)
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // [thermostatted]
    int32_t* gr_scratch = nullptr;
    int64_t gr_scratch_n = 0;
    unsigned long long* gr_counts = nullptr;
    int gr_nbins = 0;
    double* ref[BBMD_MAX_ORIGINS] = {};  // unwrapped positions by id of each time origin
    int sticky = 0;
    int device = 0;                  // CUDA device of the handle (current at creation)
    double last_dt = -1.0;           // dt of the last step call (its closing kick may be pending)
    int nsm = 1;
    int graph_gen = 0;               // bumped whenever captured launch arguments go stale
    long long tune_step = 0, tune_rebuilds = 0;  // counters at the last shape tuning
    double mean_cell = 0.0;          // mean particles per cell
    std::vector<int> shapes;         // block shapes that fit (candidates of the autotuner)
    float shape_ms[4][2] = {};       // autotuner: per kShapes entry, force and list-build ms
};

namespace {

void* dev_alloc(bbmd_sim* s, size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    void* p = nullptr;
    if (s->have_alloc) {
        p = s->alloc.alloc(bytes, s->alloc.ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) {
        s->blocks.push_back({p, bytes});
        s->bytes += (int64_t)bytes;
    }
    return p;
}

void dev_free(bbmd_sim* s, void* p) {
    if (!p) return;
    for (size_t k = 0; k < s->blocks.size(); ++k) {
        if (s->blocks[k].first == p) {
            s->bytes -= (int64_t)s->blocks[k].second;
            s->blocks.erase(s->blocks.begin() + (long)k);
            break;
        }
    }
    if (s->have_alloc)
        s->alloc.free(p, s->alloc.ctx);
    else
        cudaFree(p);
}

// Makes `dev` the calling thread's current device for the lifetime of the guard and puts
// the caller's device back afterwards, so that every call on a handle works on the device
// the handle was created on whatever device the caller has current.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
            return;
        }
        if (prev == dev) prev = -1;
        else cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
    DeviceGuard(const DeviceGuard&) = delete;
    DeviceGuard& operator=(const DeviceGuard&) = delete;
};

bbmd_status fail(bbmd_sim* s, bbmd_status code, const std::string& msg) {
    if (s) s->err = msg;
    return code;
}

bbmd_status cuda_check(bbmd_sim* s, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return BBMD_OK;
    return fail(s, BBMD_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(expr)                                                      \
    do {                                                              \
        bbmd_status _r = cuda_check(sim, (expr), #expr);              \
        if (_r != BBMD_OK) return _r;                                 \
    } while (0)

#define LAUNCHED(what)                                                \
    do {                                                              \
        bbmd_status _r = cuda_check(sim, cudaGetLastError(), what);   \
        if (_r != BBMD_OK) return _r;                                 \
    } while (0)

int fix_exponent(const double L[3]) {
    double m = std::fmax(L[0], std::fmax(L[1], L[2]));
    int e;
    std::frexp(m, &e);
    return 61 - (e - 1);
}

int bitlen(uint64_t v) {
    int b = 0;
    while (v) {
        ++b;
        v >>= 1;
    }
    return b;
}

// Cell grid rule of bbmd.h.  Returns false if some axis has fewer than 3 cells.
bool cell_grid(const double L[3], int k, double rcell, int32_t nc[3], int64_t D[3]) {
    for (int d = 0; d < 3; ++d) {
        int64_t Lf = std::llrint(std::ldexp(L[d], k));
        int64_t m = (int64_t)std::floor(L[d] / rcell);
        for (;;) {
            if (m < 3) return false;
            uint64_t q = (uint64_t)(Lf / m);
            int bl = bitlen(q);
            if (bl > 24) q &= ~((((uint64_t)1) << (bl - 24)) - 1);
            if (std::ldexp((double)q, -k) >= rcell) {
                nc[d] = (int32_t)m;
                D[d] = (int64_t)q;
                break;
            }
            --m;
        }
    }
    return true;
}

// Untruncated pair energy and derivative of Eq. lj0 / Eq. sc0.
void raw_pair(int pot, double eps, double sig, double r, double* V, double* dV) {
    double sr = sig / r, sr6 = sr * sr * sr * sr * sr * sr, sr12 = sr6 * sr6;
    if (pot == BBMD_POT_LJ) {
        *V = 4.0 * eps * (sr12 - sr6);
        *dV = 4.0 * eps * (-12.0 * sr12 + 6.0 * sr6) / r;
    } else {
        *V = 4.0 * eps * sr12;
        *dV = -48.0 * eps * sr12 / r;
    }
}

void fill_pair_table(const bbmd_params& P, PairTab& t) {
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            int k = a * 2 + b;
            double rc = P.rcut[a][b], sig = P.sigma[a][b], eps = P.eps[a][b];
            double rc2 = rc * rc;
            double R = rc + P.skin;
            double R2 = R * R;
            t.rc2[k] = rc2;
            t.R2[k] = R2;
            t.rc2lo[k] = (float)(rc2 * (1.0 - (double)kBand));
            t.rc2hi[k] = (float)(rc2 * (1.0 + (double)kBand));
            t.R2lo[k] = (float)(R2 * (1.0 - (double)kBand));
            t.R2hi[k] = (float)(R2 * (1.0 + (double)kBand));
            t.dsig2[k] = sig * sig;
            t.deps48[k] = 48.0 * eps;
            t.deps4[k] = 4.0 * eps;
            double Vc, dVc;
            raw_pair(P.potential, eps, sig, rc, &Vc, &dVc);
            t.dvshift[k] = P.shift == BBMD_SHIFT_NONE ? 0.0 : Vc;
            t.dfcut[k] = P.shift == BBMD_SHIFT_FORCE ? dVc : 0.0;
            t.drc[k] = rc;
            t.sig2[k] = (float)t.dsig2[k];
            t.sig2lo[k] = (float)(t.dsig2[k] - (double)t.sig2[k]);
            t.eps48[k] = (float)t.deps48[k];
            t.eps4[k] = (float)t.deps4[k];
            t.vshift[k] = (float)t.dvshift[k];
            t.fcut[k] = (float)t.dfcut[k];
            t.frc[k] = (float)rc;
        }
    for (int a = 0; a < 2; ++a) {
        t.mass[a] = (float)P.mass[a];
        t.dmass[a] = P.mass[a];
    }
    t.potential = P.potential;
    t.shift = P.shift;
}

bbmd_status validate(const bbmd_params* P, int64_t n, const double* box, std::string& msg) {
    if (!P || !box) return msg = "params and box are required", BBMD_ERR_ARG;
    if (n < 2 || n > 2000000000LL) return msg = "n must be in [2, 2e9]", BBMD_ERR_ARG;
    for (int d = 0; d < 3; ++d)
        if (!(box[d] >= 1.0 && box[d] < 1e9)) return msg = "box sides must be in [1, 1e9)", BBMD_ERR_ARG;
    if (P->potential != BBMD_POT_LJ && P->potential != BBMD_POT_SOFT) return msg = "potential", BBMD_ERR_ARG;
    if (P->shift < 0 || P->shift > 2) return msg = "shift", BBMD_ERR_ARG;
    if (P->precision != BBMD_PREC_MIXED && P->precision != BBMD_PREC_FP64) return msg = "precision", BBMD_ERR_ARG;
    if (P->nbr_mode != BBMD_NBR_VERLET && P->nbr_mode != BBMD_NBR_CELL) return msg = "nbr_mode", BBMD_ERR_ARG;
    if (!(P->skin >= 0.0 && P->skin < 10.0)) return msg = "skin", BBMD_ERR_ARG;
    for (int a = 0; a < 2; ++a) {
        if (!(P->mass[a] > 0.0)) return msg = "mass must be > 0", BBMD_ERR_ARG;
        for (int b = 0; b < 2; ++b) {
            if (!(P->rcut[a][b] > 0.0) || !(P->sigma[a][b] > 0.0) || !(P->eps[a][b] >= 0.0))
                return msg = "rcut, sigma > 0 and eps >= 0 required", BBMD_ERR_ARG;
            if (P->rcut[a][b] != P->rcut[b][a] || P->sigma[a][b] != P->sigma[b][a] ||
                P->eps[a][b] != P->eps[b][a])
                return msg = "pair tables must be symmetric", BBMD_ERR_ARG;
        }
    }
    if (P->list_capacity < 0 || P->list_capacity > 4096) return msg = "list_capacity", BBMD_ERR_ARG;
    if (P->stencil_capacity < 0 || P->stencil_capacity > 65000) return msg = "stencil_capacity", BBMD_ERR_ARG;
    if (P->block_z != 0 && P->block_z != 1 && P->block_z != 2 && P->block_z != 4 && P->block_z != 8)
        return msg = "block_z must be 0 (autotune), 1, 2, 4 or 8", BBMD_ERR_ARG;
    if (!(P->init_jitter >= 0.0 && P->init_jitter < 1e6)) return msg = "init_jitter", BBMD_ERR_ARG;
    return BBMD_OK;
}

bool all_finite(const double* a, int64_t m) {
    if (!a) return true;
    for (int64_t i = 0; i < m; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

// Staged capacity of one block region for shape bz (user capacity, else from the mean
// cell occupancy with 15 % headroom), rounded to 32.
int shape_smax(const bbmd_sim* sim, int bz) {
    int smax = sim->P.stencil_capacity > 0
                   ? sim->P.stencil_capacity
                   : (int)((double)region_cells_of(bz) * sim->mean_cell * 1.15 + 160.0);
    return (smax + 31) / 32 * 32;
}

// The staged region and its sentinel record must fit in shared memory as 32-byte records
// (the FP64 form, and the FP64 energy pass of mixed precision) and its offsets in uint16
// (the sentinel is smax itself).
bool shape_fits(const bbmd_sim* sim, int bz) {
    const int smax = shape_smax(sim, bz);
    const size_t bytes = (size_t)(smax + 1) * 32;
    return smax <= 65000 && bytes <= 200 * 1024;
}

// Select block shape bz: geometry, staged capacity and the grids of the block kernels.
void apply_shape(bbmd_sim* sim, int bz) {
    DevSim& D = sim->d;
    D.block_z = bz;
    D.region_cells = region_cells_of(bz);
    D.smax = shape_smax(sim, bz);
    const int bxy = block_xy_of(bz), bzc = block_zc_of(bz);
    D.nblocks = (int64_t)((D.nc[0] + bxy - 1) / bxy) * ((D.nc[1] + bxy - 1) / bxy) *
                ((D.nc[2] + bzc - 1) / bzc);
    int64_t g = (int64_t)sim->nsm * force_blocks_per_sm(D);
    if (g > D.nblocks) g = D.nblocks;
    if (g > kMaxPartials) g = kMaxPartials;
    D.grid_cell = (int32_t)(g > 0 ? g : 1);
    g = (int64_t)sim->nsm * list_blocks_per_sm(D);
    if (g > D.nblocks) g = D.nblocks;
    D.grid_list = (int32_t)(g > 0 ? g : 1);
}

bbmd_status rebuild_now(bbmd_sim* sim);
bbmd_status refresh_forces_and_K(bbmd_sim* sim);
void finish_velocities(bbmd_sim* sim);
void free_graphs(bbmd_sim* sim);

// A list build cut some lists at the capacity (Verlet mode).  The steps since then took
// their forces from the cell stencil, which is exact.  Grow the capacity to the longest
// list seen plus an eighth (at most 4096 entries), rebuild the lists and recompute the
// forces.  If the cap is reached, the status bit stays and the caller reports the overflow.
bbmd_status grow_lists(bbmd_sim* sim) {
    DevSim& D = sim->d;
    if (D.nbr_mode != BBMD_NBR_VERLET) return BBMD_OK;
    for (int attempt = 0; attempt < 8; ++attempt) {
        int st = 0, longest = 0;
        CK(cudaMemcpyAsync(&st, &D.sc->status, sizeof(int), cudaMemcpyDeviceToHost, sim->st));
        CK(cudaMemcpyAsync(&longest, &D.sc->max_len, sizeof(int), cudaMemcpyDeviceToHost, sim->st));
        CK(cudaStreamSynchronize(sim->st));
        const int cap = D.lcap8 * 8;
        if (!(st & ST_LIST_OVERFLOW) || (st & ST_STENCIL_OVERFLOW) || cap >= 4096) return BBMD_OK;
        int want = std::max(longest + longest / 8 + 8, cap + 8);
        want = std::min(4096, (want + 7) / 8 * 8);
        uint16_t* grown = (uint16_t*)dev_alloc(sim, (size_t)(want / 8) * (size_t)D.npad * 16);
        if (!grown) return fail(sim, BBMD_ERR_OOM, "growing the Verlet lists");
        dev_free(sim, D.list);
        D.list = grown;
        D.lcap8 = want / 8;
        free_graphs(sim);  // the captured kernels hold the old list
        const int cleared = st & ~ST_LIST_OVERFLOW;
        CK(cudaMemcpyAsync(&D.sc->status, &cleared, sizeof(int), cudaMemcpyHostToDevice, sim->st));
        CK(cudaStreamSynchronize(sim->st));  // `cleared` lives on this stack frame
        finish_velocities(sim);  // the pending kick used the forces about to be recomputed
        rebuild_now(sim);
        refresh_forces_and_K(sim);
    }
    return BBMD_OK;
}

// The status word: grow cut lists if needed, then report the sticky bits.  `known`: the
// status word the caller has just read after synchronising (skips two round trips unless
// lists were cut), or -1.
bbmd_status read_status(bbmd_sim* sim, int known = -1) {
    int st = known;
    if (known < 0 || (known & ST_LIST_OVERFLOW)) {
        bbmd_status g = grow_lists(sim);
        if (g != BBMD_OK) return g;
        CK(cudaMemcpyAsync(&st, &sim->d.sc->status, sizeof(int), cudaMemcpyDeviceToHost, sim->st));
        CK(cudaStreamSynchronize(sim->st));
    }
    sim->sticky |= st;
    if (sim->sticky & (ST_LIST_OVERFLOW | ST_STENCIL_OVERFLOW))
        return fail(sim, BBMD_ERR_LIST_OVERFLOW,
                    "a Verlet list or staged stencil exceeded its capacity (raise list_capacity / "
                    "stencil_capacity)");
    if (sim->sticky & (ST_NONFINITE | ST_VEL_RANGE))
        return fail(sim, BBMD_ERR_NUMERIC, "non-finite force or velocity beyond the fixed-point range");
    if (sim->sticky & ST_TIMEOUT) return fail(sim, BBMD_ERR_TIMEOUT, "a bounded device wait gave up");
    return BBMD_OK;
}

void enqueue_rebuild(bbmd_sim* sim) {
    launch_rebuild_chain(sim->d, sim->st);
    launch_list_build(sim->d, sim->st);
}

// Force a rebuild now: set the flag, run the chain and clear it.
bbmd_status rebuild_now(bbmd_sim* sim) {
    int one = 1;
    CK(cudaMemcpyAsync(&sim->d.sc->rebuild, &one, sizeof(int), cudaMemcpyHostToDevice, sim->st));
    enqueue_rebuild(sim);
    launch_clear_rebuild(sim->d, sim->st);
    LAUNCHED("rebuild");
    return BBMD_OK;
}

// Block-shape autotuner, run once at creation on the system's own initial state (cells
// already sorted): for every candidate shape, time one list build (Verlet mode) and one
// force evaluation with CUDA events, after an untimed launch of each, over the first blocks
// of the box (up to 131072 cells; the cost per cell is what is compared, scaled to the
// whole box); keep the shape of least force + list / 4 (a rebuild about every four steps).
// A shape whose staged region or lists overflow is dropped.  The lists of the chosen shape
// are rebuilt at the end, over the whole box.
bbmd_status autotune_shape(bbmd_sim* sim, float rebuild_rate = 0.25f) {
    DevSim& D = sim->d;
    const bool verlet = D.nbr_mode == BBMD_NBR_VERLET;
    cudaEvent_t ev[4];
    for (auto& e : ev) CK(cudaEventCreate(&e));
    int status0 = 0;
    CK(cudaMemcpyAsync(&status0, &D.sc->status, sizeof(int), cudaMemcpyDeviceToHost, sim->st));
    CK(cudaStreamSynchronize(sim->st));
    int best = -1;
    float best_cost = 0.f;
    const int one = 1, zero = 0;
    const int64_t target_cells = std::min<int64_t>(D.ncell, 131072);
    for (int bz : sim->shapes) {
        apply_shape(sim, bz);
        // the timed launches cover the first nb blocks only
        DevSim Dt = D;
        const int64_t cpb = block_cells_of(bz);
        Dt.nblocks = std::min<int64_t>(D.nblocks, (target_cells + cpb - 1) / cpb);
        Dt.grid_cell = (int32_t)std::min<int64_t>(Dt.grid_cell, Dt.nblocks);
        Dt.grid_list = (int32_t)std::min<int64_t>(Dt.grid_list, Dt.nblocks);
        const double scale = (double)D.nblocks / (double)Dt.nblocks;
        CK(cudaMemcpyAsync(&D.sc->rebuild, &one, sizeof(int), cudaMemcpyHostToDevice, sim->st));
        if (verlet) launch_list_build(Dt, sim->st);
        CK(cudaEventRecord(ev[0], sim->st));
        if (verlet) launch_list_build(Dt, sim->st);
        CK(cudaEventRecord(ev[1], sim->st));
        CK(cudaMemcpyAsync(&D.sc->rebuild, &zero, sizeof(int), cudaMemcpyHostToDevice, sim->st));
        launch_force(Dt, sim->st, false, false);
        CK(cudaEventRecord(ev[2], sim->st));
        launch_force(Dt, sim->st, false, false);
        CK(cudaEventRecord(ev[3], sim->st));
        LAUNCHED("autotune");
        int st = 0;
        CK(cudaMemcpyAsync(&st, &D.sc->status, sizeof(int), cudaMemcpyDeviceToHost, sim->st));
        CK(cudaStreamSynchronize(sim->st));
        float tl = 0.f, tf = 0.f;
        CK(cudaEventElapsedTime(&tl, ev[0], ev[1]));
        CK(cudaEventElapsedTime(&tf, ev[2], ev[3]));
        tf = (float)(tf * scale);
        tl = (float)(tl * scale);
        int k = 0;
        while (kShapes[k] != bz) ++k;
        sim->shape_ms[k][0] = tf;
        sim->shape_ms[k][1] = tl;
        if (st & (ST_LIST_OVERFLOW | ST_STENCIL_OVERFLOW)) {
            // drop the shape and restore the status word
            CK(cudaMemcpyAsync(&D.sc->status, &status0, sizeof(int), cudaMemcpyHostToDevice, sim->st));
            continue;
        }
        const float cost = tf + (verlet ? rebuild_rate * tl : 0.f);
        if (best < 0 || cost < best_cost) {
            best = bz;
            best_cost = cost;
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    if (best < 0) best = sim->shapes[0];  // every shape overflowed: keep the first, report it
    apply_shape(sim, best);
    CK(cudaMemcpyAsync(&D.sc->rebuild, &one, sizeof(int), cudaMemcpyHostToDevice, sim->st));
    if (verlet) launch_list_build(D, sim->st);
    CK(cudaMemcpyAsync(&D.sc->rebuild, &zero, sizeof(int), cudaMemcpyHostToDevice, sim->st));
    LAUNCHED("autotune rebuild");
    return BBMD_OK;
}

bbmd_status refresh_forces_and_K(bbmd_sim* sim) {
    launch_force(sim->d, sim->st, false, false);
    launch_state_sums(sim->d, sim->st);
    launch_reduce_partials(sim->d, sim->st, 4, sim->dout);
    LAUNCHED("forces");
    // sc->K <- KE of the stored velocities
    CK(cudaMemcpyAsync(&sim->d.sc->K, sim->dout, sizeof(double), cudaMemcpyDeviceToDevice, sim->st));
    return BBMD_OK;
}

void free_graphs(bbmd_sim* sim) {
    ++sim->graph_gen;
    for (auto& g : sim->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

// Start of a step call: the closing half kick a previous call left pending is carried into
// this call's first update when dt is unchanged; otherwise it is applied now.
void begin_call(bbmd_sim* sim, int64_t nsteps, double dt, const bbmd_thermostat* th) {
    if (dt != sim->last_dt) launch_finish(sim->d, sim->st);
    launch_begin(sim->d, sim->st, nsteps, dt, th);
    sim->last_dt = dt;
}

// Apply a pending closing half kick to the stored velocities (before velocities are read
// out or replaced, or positions move outside a step).
void finish_velocities(bbmd_sim* sim) { launch_finish(sim->d, sim->st); }

bbmd_status build_graph(bbmd_sim* sim, int nh) {
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(sim->st, cudaStreamCaptureModeThreadLocal));
    launch_integrate(sim->d, sim->st);
    launch_check(sim->d, sim->st);
    enqueue_rebuild(sim);
    launch_force(sim->d, sim->st, false, nh != 0);
    launch_finalize(sim->d, sim->st, nh != 0);
    cudaError_t e = cudaStreamEndCapture(sim->st, &g);
    CK(e);
    e = cudaGraphInstantiate(&sim->graph[nh], g, 0);
    cudaGraphDestroy(g);
    CK(e);
    return BBMD_OK;
}

}  // namespace

extern "C" {

bbmd_status bbmd_create(const bbmd_params* params, int64_t n, const double box[3],
                        const uint8_t* species, const double* pos, const double* vel, double T0,
                        uint64_t seed, void* stream, const bbmd_alloc* alloc, bbmd_sim** out) {
    if (!out) return BBMD_ERR_ARG;
    *out = nullptr;
    std::string msg;
    bbmd_status vs = validate(params, n, box, msg);
    if (vs != BBMD_OK) {
        std::fprintf(stderr, "bbmd_create: %s\n", msg.c_str());
        return vs;
    }
    if (!species) return BBMD_ERR_ARG;
    for (int64_t i = 0; i < n; ++i)
        if (species[i] > 1) {
            std::fprintf(stderr, "bbmd_create: species labels must be 0 or 1\n");
            return BBMD_ERR_ARG;
        }
    if (!(T0 >= 0.0)) return BBMD_ERR_ARG;
    if (!all_finite(pos, 3 * n) || !all_finite(vel, 3 * n)) {
        std::fprintf(stderr, "bbmd_create: non-finite positions or velocities\n");
        return BBMD_ERR_ARG;
    }
    int m_fcc = 0;
    if (!pos) {
        m_fcc = (int)std::llround(std::cbrt((double)n / 4.0));
        if (4LL * m_fcc * m_fcc * m_fcc != n) return BBMD_ERR_ARG;
    }
    bbmd_sim* sim = new bbmd_sim();
    sim->P = *params;
    if (cudaGetDevice(&sim->device) != cudaSuccess) {
        cudaGetLastError();
        delete sim;
        return BBMD_ERR_CUDA;
    }
    sim->st = (cudaStream_t)stream;
    if (!sim->st) {
        if (cudaStreamCreateWithFlags(&sim->st, cudaStreamNonBlocking) != cudaSuccess) {
            delete sim;
            return BBMD_ERR_CUDA;
        }
        sim->own_stream = true;
    }
    if (alloc && alloc->alloc && alloc->free) {
        sim->alloc = *alloc;
        sim->have_alloc = true;
    }
    for (int d = 0; d < 3; ++d) sim->box[d] = box[d];
    DevSim& D = sim->d;
    std::memset(&D, 0, sizeof(D));
    D.n = n;
    D.npad = (n + 63) / 64 * 64;
    D.kexp = fix_exponent(box);
    D.sx = std::ldexp(1.0f, -D.kexp);
    D.sxd = std::ldexp(1.0, -D.kexp);
    for (int d = 0; d < 3; ++d) D.Lfix[d] = std::llrint(std::ldexp(box[d], D.kexp));
    double rcmax = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) rcmax = std::fmax(rcmax, params->rcut[a][b]);
    double rcell = rcmax + params->skin;
    if (!cell_grid(box, D.kexp, rcell, D.nc, D.D)) {
        bbmd_destroy(sim);
        return BBMD_ERR_BOX_TOO_SMALL;
    }
    int64_t ncell = (int64_t)D.nc[0] * D.nc[1] * D.nc[2];
    if (ncell > 0x7fffffffLL / 2) {
        bbmd_destroy(sim);
        return BBMD_ERR_ARG;
    }
    D.ncell = (int32_t)ncell;
    D.nbr_mode = params->nbr_mode;
    D.precision = params->precision;
    fill_pair_table(*params, D.pt);
    for (int k = 0; k < 4; ++k)
        D.pt.rcfix[k] = (long long)std::ceil(std::ldexp(D.pt.drc[k], D.kexp));
    double half = 0.5 * params->skin;
    D.disp2 = (float)(half * half * (1.0 - 1e-4));
    D.disp_thr = (float)(params->skin * (1.0 - 1e-4));
    {
        // cells two apart along an axis are more than one cell side apart
        double dmin = std::ldexp((double)std::min(D.D[0], std::min(D.D[1], D.D[2])), -D.kexp);
        D.disp_far = (float)((dmin - rcmax) * (1.0 - 1e-4));
    }
    int lcap = params->list_capacity > 0 ? params->list_capacity : 160;
    D.lcap8 = (lcap + 7) / 8;
    double V = box[0] * box[1] * box[2];
    double cellvol = std::ldexp((double)D.D[0], -D.kexp) * std::ldexp((double)D.D[1], -D.kexp) *
                     std::ldexp((double)D.D[2], -D.kexp);
    double mean = (double)n / V * cellvol;
    for (int d = 0; d < 3; ++d) D.halfL[d] = (float)(0.5 * box[d]);
    if (!prepare_force_kernels()) {
        cudaGetLastError();
        std::fprintf(stderr, "bbmd_create: could not configure kernel shared memory\n");
        bbmd_destroy(sim);
        return BBMD_ERR_CUDA;
    }
    // device properties and grids
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, sim->device);
    if (nsm <= 0) nsm = 1;
    // per-particle grid-stride kernels: 8 CTAs per SM, fewer for a small system
    D.grid_part = (int32_t)std::min<int64_t>((int64_t)nsm * 8, std::max<int64_t>(1, (n + 255) / 256));
    sim->nsm = nsm;
    sim->mean_cell = mean;
    // block shapes that fit this system (all of them are tried at the end of creation unless
    // params->block_z fixes one)
    for (int bz : kShapes) {
        if (params->block_z != 0 && bz != params->block_z) continue;
        // a block's own cells are distinct cells of the box (the staged region wraps the
        // box at most once)
        if (block_xy_of(bz) > D.nc[0] || block_xy_of(bz) > D.nc[1] || block_zc_of(bz) > D.nc[2])
            continue;
        if (!shape_fits(sim, bz)) continue;
        sim->shapes.push_back(bz);
    }
    if (sim->shapes.empty()) {
        std::fprintf(stderr, "bbmd_create: no block shape fits (staged region beyond shared "
                             "memory, or the block larger than the cells along an axis)\n");
        bbmd_destroy(sim);
        return BBMD_ERR_ARG;
    }
    apply_shape(sim, sim->shapes[0]);

    // memory plan
    const int64_t np = D.npad;
    bool ok = true;
    auto A = [&](size_t bytes) -> void* {
        void* p = dev_alloc(sim, bytes);
        if (!p) ok = false;
        return p;
    };
    D.x = (uint64_t*)A(3 * np * 8);
    D.v = (int64_t*)A(3 * np * 8);
    D.img = (int32_t*)A(3 * np * 4);
    D.id = (int32_t*)A(np * 4);
    D.sp = (uint8_t*)A(np);
    D.x2 = (uint64_t*)A(3 * np * 8);
    D.v2 = (int64_t*)A(3 * np * 8);
    D.img2 = (int32_t*)A(3 * np * 4);
    D.id2 = (int32_t*)A(np * 4);
    D.sp2 = (uint8_t*)A(np);
    D.rel = (float4*)A(np * 16);
    D.relb = (float4*)A(np * 16);
    D.F = (float4*)A(np * 16);
    if (params->precision == BBMD_PREC_FP64) D.Fd = (double*)A(3 * np * 8);
    D.ud = (double*)A(np * 8);
    D.key = (int32_t*)A(np * 4);
    D.perm = (int32_t*)A(np * 4);
    D.perm_tmp = (int32_t*)A(np * 4);
    D.count = (int32_t*)A((ncell + 1) * 4);
    D.cursor = (int32_t*)A((ncell + 1) * 4);
    D.cell_start = (int32_t*)A((ncell + 1) * 4);
    D.scan_part = (int32_t*)A(((ncell + 8191) / 8192 + 1) * 4);
    if (params->nbr_mode == BBMD_NBR_VERLET) D.list = (uint16_t*)A((size_t)D.lcap8 * np * 16);
    D.rows = (uint16_t*)A(np * 2);
    D.partials = (double*)A((size_t)8 * kMaxPartials * 8);
    D.disp = (float*)A(np * 4);
    D.mtop = (float2*)A((size_t)ncell * 8);
    D.sc = (DevScalars*)A(sizeof(DevScalars));
    sim->dout = (double*)A(64 * 8);
    if (!ok) {
        bbmd_destroy(sim);
        return BBMD_ERR_OOM;
    }
    if (cudaMemsetAsync(D.sc, 0, sizeof(DevScalars), sim->st) != cudaSuccess ||
        cudaMemsetAsync(D.rows, 0, np * 2, sim->st) != cudaSuccess ||
        cudaMemsetAsync(D.img, 0, 3 * np * 4, sim->st) != cudaSuccess ||
        cudaMemsetAsync(D.disp, 0, np * 4, sim->st) != cudaSuccess) {
        bbmd_destroy(sim);
        return BBMD_ERR_CUDA;
    }

    // initial state (id order), through temporary device buffers
    bbmd_status rc = BBMD_OK;
    double* tpos = nullptr;
    double* tvel = nullptr;
    if (cudaMemcpyAsync(D.sp2, species, (size_t)n, cudaMemcpyHostToDevice, sim->st) != cudaSuccess)
        rc = BBMD_ERR_CUDA;
    if (rc == BBMD_OK && pos) {
        tpos = (double*)dev_alloc(sim, 3 * n * 8);
        if (!tpos) rc = BBMD_ERR_OOM;
        else if (cudaMemcpyAsync(tpos, pos, 3 * n * 8, cudaMemcpyHostToDevice, sim->st) != cudaSuccess)
            rc = BBMD_ERR_CUDA;
    }
    if (rc == BBMD_OK && vel) {
        tvel = (double*)dev_alloc(sim, 3 * n * 8);
        if (!tvel) rc = BBMD_ERR_OOM;
        else if (cudaMemcpyAsync(tvel, vel, 3 * n * 8, cudaMemcpyHostToDevice, sim->st) != cudaSuccess)
            rc = BBMD_ERR_CUDA;
    }
    if (rc == BBMD_OK) {
        launch_pack_state(D, sim->st, tpos, tvel, nullptr, false);
        if (!pos) launch_init_fcc(D, sim->st, m_fcc, params->init_jitter, seed);
        if (!vel) {
            double* tmp = (double*)dev_alloc(sim, (3 * n + 16) * 8);
            if (!tmp) rc = BBMD_ERR_OOM;
            else {
                launch_init_mb(D, sim->st, T0, seed, tmp);
                cudaStreamSynchronize(sim->st);
                dev_free(sim, tmp);
            }
        }
    }
    if (rc == BBMD_OK && cudaStreamSynchronize(sim->st) != cudaSuccess) rc = BBMD_ERR_CUDA;
    dev_free(sim, tpos);
    dev_free(sim, tvel);
    if (rc == BBMD_OK) rc = rebuild_now(sim);
    if (rc == BBMD_OK) rc = grow_lists(sim);  // lists longer than the capacity asked for
    if (rc == BBMD_OK && sim->shapes.size() > 1) rc = autotune_shape(sim);
    if (rc == BBMD_OK) rc = refresh_forces_and_K(sim);
    if (rc == BBMD_OK) rc = read_status(sim);
    if (rc != BBMD_OK) {
        std::fprintf(stderr, "bbmd_create: %s\n", sim->err.c_str());
        bbmd_destroy(sim);
        return rc;
    }
    *out = sim;
    return BBMD_OK;
}

void bbmd_destroy(bbmd_sim* sim) {
    if (!sim) return;
    DeviceGuard dg(sim->device);
    if (sim->st) cudaStreamSynchronize(sim->st);
    else cudaDeviceSynchronize();
    free_graphs(sim);
    while (!sim->blocks.empty()) dev_free(sim, sim->blocks.back().first);
    if (sim->own_stream) cudaStreamDestroy(sim->st);
    delete sim;
}

bbmd_status bbmd_step_profiled(bbmd_sim* sim, int64_t nsteps, double dt, const bbmd_thermostat* th,
                               double* ms, int64_t* rebuilds) {
    if (!sim) return BBMD_ERR_ARG;
    DeviceGuard dg(sim->device);
    if (nsteps < 0 || nsteps > 0x7fffffff || !(dt > 0.0) || !(dt < 1.0))
        return fail(sim, BBMD_ERR_ARG, "nsteps in [0, 2^31) and dt in (0, 1) required");
    int nh = th && th->kind == BBMD_THERMO_NH;
    if (nh && !(th->T_start > 0.0 && th->T_end > 0.0 && th->tau > 0.0))
        return fail(sim, BBMD_ERR_ARG, "Nose-Hoover needs T_start, T_end, tau > 0");
    cudaEvent_t ev[BBMD_PHASE_COUNT + 1];
    for (auto& e : ev) CK(cudaEventCreate(&e));
    double acc[BBMD_PHASE_COUNT] = {0, 0, 0, 0, 0};
    DevScalars scl0;
    CK(cudaMemcpyAsync(&scl0, sim->d.sc, sizeof(scl0), cudaMemcpyDeviceToHost, sim->st));
    begin_call(sim, nsteps, dt, nh ? th : nullptr);
    for (int64_t k = 0; k < nsteps; ++k) {
        CK(cudaEventRecord(ev[0], sim->st));
        launch_integrate(sim->d, sim->st);
        launch_check(sim->d, sim->st);
        CK(cudaEventRecord(ev[1], sim->st));
        launch_rebuild_chain(sim->d, sim->st);
        CK(cudaEventRecord(ev[2], sim->st));
        launch_list_build(sim->d, sim->st);
        CK(cudaEventRecord(ev[3], sim->st));
        launch_force(sim->d, sim->st, false, nh != 0);
        CK(cudaEventRecord(ev[4], sim->st));
        launch_finalize(sim->d, sim->st, nh != 0);
        CK(cudaEventRecord(ev[5], sim->st));
        LAUNCHED("profiled step");
        CK(cudaEventSynchronize(ev[5]));
        for (int q = 0; q < BBMD_PHASE_COUNT; ++q) {
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, ev[q], ev[q + 1]));
            acc[q] += t;
        }
    }
    DevScalars scl1;
    CK(cudaMemcpyAsync(&scl1, sim->d.sc, sizeof(scl1), cudaMemcpyDeviceToHost, sim->st));
    CK(cudaStreamSynchronize(sim->st));
    for (auto& e : ev) cudaEventDestroy(e);
    if (ms)
        for (int q = 0; q < BBMD_PHASE_COUNT; ++q) ms[q] = acc[q];
    if (rebuilds) *rebuilds = scl1.n_rebuilds - scl0.n_rebuilds;
    return read_status(sim);
}

bbmd_status bbmd_step(bbmd_sim* sim, int64_t nsteps, double dt, const bbmd_thermostat* th) {
    if (!sim) return BBMD_ERR_ARG;
    DeviceGuard dg(sim->device);
    if (nsteps < 0 || nsteps > 0x7fffffff || !(dt > 0.0) || !(dt < 1.0))
        return fail(sim, BBMD_ERR_ARG, "nsteps in [0, 2^31) and dt in (0, 1) required");
    int nh = 0;
    if (th) {
        if (th->kind == BBMD_THERMO_NH) {
            if (!(th->T_start > 0.0 && th->T_end > 0.0 && th->tau > 0.0))
                return fail(sim, BBMD_ERR_ARG, "Nose-Hoover needs T_start, T_end, tau > 0");
            nh = 1;
        } else if (th->kind != BBMD_THERMO_NVE) {
            return fail(sim, BBMD_ERR_ARG, "thermostat kind");
        }
    }
    if (nsteps == 0) return BBMD_OK;
    if (!sim->graph[nh]) {
        bbmd_status r = build_graph(sim, nh);
        if (r != BBMD_OK) return r;
    }
    begin_call(sim, nsteps, dt, nh ? th : nullptr);
    LAUNCHED("begin");
    for (int64_t k = 0; k < nsteps; ++k) CK(cudaGraphLaunch(sim->graph[nh], sim->st));
    return BBMD_OK;
}

bbmd_status bbmd_observe(bbmd_sim* sim, uint32_t mask, const bbmd_obs_args* args, bbmd_obs* out) {
    if (!sim || !out) return BBMD_ERR_ARG;
    DeviceGuard dg(sim->device);
    int nbins = args && args->nbins > 0 ? args->nbins : 500;
    double rmax = args && args->rmax > 0.0 ? args->rmax : 5.0;
    double kv = args && args->k > 0.0 ? args->k : 7.25;
    if (nbins > 4096) return fail(sim, BBMD_ERR_ARG, "nbins <= 4096");
    DevSim& D = sim->d;
    // kinetic energy and momentum
    launch_state_sums(D, sim->st);
    launch_reduce_partials(D, sim->st, 4, sim->dout);
    if (mask & (BBMD_OBS_ENERGY | BBMD_OBS_VIRIAL)) {
        launch_force(D, sim->st, true, false);
        launch_reduce_partials(D, sim->st, -3, sim->dout + 8);
    }
    const int origin = args ? args->origin : 0;
    if (origin < 0 || origin >= BBMD_MAX_ORIGINS)
        return fail(sim, BBMD_ERR_ARG, "origin must be in [0, BBMD_MAX_ORIGINS)");
    if (mask & BBMD_OBS_SET_REF) {
        if (!sim->ref[origin]) {
            sim->ref[origin] = (double*)dev_alloc(sim, 3 * D.n * 8);
            if (!sim->ref[origin]) return fail(sim, BBMD_ERR_OOM, "reference positions");
        }
        launch_set_ref(D, sim->st, sim->ref[origin]);
    }
    if (mask & (BBMD_OBS_MSD | BBMD_OBS_FS)) {
        if (!sim->ref[origin]) return fail(sim, BBMD_ERR_STATE, "MSD/FS need SET_REF of this origin first");
        launch_msd_fs(D, sim->st, sim->ref[origin], kv, sim->dout + 16);
    }
    std::vector<unsigned long long> counts;
    if (mask & BBMD_OBS_GR) {
        if (!sim->gr_counts || sim->gr_nbins < nbins) {
            dev_free(sim, sim->gr_counts);
            sim->gr_counts = (unsigned long long*)dev_alloc(sim, (size_t)4 * nbins * 8);
            sim->gr_nbins = nbins;
        }
        int64_t ncg = 1;
        for (int d = 0; d < 3; ++d) {
            int m = (int)std::floor(sim->box[d] / rmax);
            ncg *= m < 1 ? 1 : m;
        }
        int64_t need = 2 * D.n + 3 * (ncg + 1);
        if (sim->gr_scratch_n < need) {
            dev_free(sim, sim->gr_scratch);
            sim->gr_scratch = (int32_t*)dev_alloc(sim, (size_t)need * 4);
            sim->gr_scratch_n = sim->gr_scratch ? need : 0;
        }
        if (!sim->gr_counts || !sim->gr_scratch) return fail(sim, BBMD_ERR_OOM, "g(r) scratch");
        if (launch_gr(D, sim->st, nbins, rmax, sim->gr_counts, sim->gr_scratch, nullptr,
                      sim->gr_scratch_n) != 0)
            return fail(sim, BBMD_ERR_STATE, "g(r) scratch too small");
        counts.resize((size_t)4 * nbins);
        CK(cudaMemcpyAsync(counts.data(), sim->gr_counts, counts.size() * 8, cudaMemcpyDeviceToHost,
                           sim->st));
    }
    LAUNCHED("observe");
    double h[32];
    DevScalars scl;
    CK(cudaMemcpyAsync(h, sim->dout, sizeof(h), cudaMemcpyDeviceToHost, sim->st));
    CK(cudaMemcpyAsync(&scl, D.sc, sizeof(scl), cudaMemcpyDeviceToHost, sim->st));
    CK(cudaStreamSynchronize(sim->st));
    bbmd_status rs = read_status(sim, scl.status);
    if (rs != BBMD_OK) return rs;
    double Vol = sim->box[0] * sim->box[1] * sim->box[2];
    double g = (double)(3 * D.n - 3);
    out->ke = h[0];
    out->momentum[0] = h[1];
    out->momentum[1] = h[2];
    out->momentum[2] = h[3];
    out->temperature = 2.0 * h[0] / g;
    out->step = scl.step;
    out->n_rebuilds = scl.n_rebuilds;
    out->xi = scl.xi;
    out->eta = scl.eta;
    if (mask & (BBMD_OBS_ENERGY | BBMD_OBS_VIRIAL)) {
        out->pe = h[9];
        out->virial = h[10];
        out->pressure = (2.0 * h[0] + h[10]) / (3.0 * Vol);
        double E = h[0] + h[9];
        if (scl.kind == BBMD_THERMO_NH && scl.tau > 0.0 && scl.T_last > 0.0) {
            double Q = g * scl.T_last * scl.tau * scl.tau;
            E += 0.5 * Q * scl.xi * scl.xi + g * scl.T_last * scl.eta;
        }
        out->conserved = E;
    }
    if (mask & (BBMD_OBS_MSD | BBMD_OBS_FS)) {
        for (int a = 0; a < 2; ++a) {
            double cnt = h[16 + 4 + a];
            out->msd[a] = cnt > 0 ? h[16 + a] / cnt : 0.0;
            out->fs[a] = cnt > 0 ? h[16 + 2 + a] / cnt : 0.0;
        }
    }
    if (mask & BBMD_OBS_GR) {
        double Ns[2] = {0.0, 0.0};
        // species counts from the pair totals are not exact for empty shells; count directly
        std::vector<uint8_t> spc((size_t)D.n);
        CK(cudaMemcpy(spc.data(), D.sp, (size_t)D.n, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < D.n; ++i) Ns[spc[(size_t)i]] += 1.0;
        double dr = rmax / (double)nbins;
        const double pi = 3.14159265358979323846;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                double nb = Ns[b] - (a == b ? 1.0 : 0.0);
                for (int q = 0; q < nbins; ++q) {
                    size_t k = (size_t)(a * 2 + b) * nbins + q;
                    if (out->gr_counts) out->gr_counts[k] = counts[k];
                    if (out->gr) {
                        double r0 = dr * (double)q, r1 = dr * (double)(q + 1);
                        double shell = (4.0 * pi / 3.0) * (r1 * r1 * r1 - r0 * r0 * r0);
                        double den = Ns[a] * nb * shell;
                        out->gr[k] = den > 0.0 ? Vol * (double)counts[k] / den : 0.0;
                    }
                }
            }
    }
    return BBMD_OK;
}

bbmd_status bbmd_minimize(bbmd_sim* sim, int64_t nsteps, double hmax, double dmax) {
    if (!sim || nsteps < 0 || !(hmax > 0.0) || !(dmax > 0.0)) return BBMD_ERR_ARG;
    DeviceGuard dg(sim->device);
    finish_velocities(sim);
    for (int64_t k = 0; k < nsteps; ++k) {
        launch_force(sim->d, sim->st, false, false);
        launch_sd_step(sim->d, sim->st, hmax, dmax);
        enqueue_rebuild(sim);
        launch_clear_rebuild(sim->d, sim->st);
    }
    LAUNCHED("minimize");
    launch_force(sim->d, sim->st, false, false);
    LAUNCHED("minimize forces");
    return read_status(sim);
}

bbmd_status bbmd_get_state(bbmd_sim* sim, double* pos, double* vel, int32_t* image) {
    if (!sim) return BBMD_ERR_ARG;
    DeviceGuard dg(sim->device);
    finish_velocities(sim);
    const int64_t n = sim->d.n;
    double* tp = pos ? (double*)dev_alloc(sim, 3 * n * 8) : nullptr;
    double* tv = vel ? (double*)dev_alloc(sim, 3 * n * 8) : nullptr;
    int32_t* ti = image ? (int32_t*)dev_alloc(sim, 3 * n * 4) : nullptr;
    bbmd_status rc = BBMD_OK;
    if ((pos && !tp) || (vel && !tv) || (image && !ti)) rc = fail(sim, BBMD_ERR_OOM, "get_state");
    if (rc == BBMD_OK) {
        launch_unpack_state(sim->d, sim->st, tp, tv, ti);
        rc = cuda_check(sim, cudaGetLastError(), "unpack");
    }
    if (rc == BBMD_OK && pos)
        rc = cuda_check(sim, cudaMemcpyAsync(pos, tp, 3 * n * 8, cudaMemcpyDeviceToHost, sim->st), "D2H");
    if (rc == BBMD_OK && vel)
        rc = cuda_check(sim, cudaMemcpyAsync(vel, tv, 3 * n * 8, cudaMemcpyDeviceToHost, sim->st), "D2H");
    if (rc == BBMD_OK && image)
        rc = cuda_check(sim, cudaMemcpyAsync(image, ti, 3 * n * 4, cudaMemcpyDeviceToHost, sim->st), "D2H");
    if (rc == BBMD_OK) rc = cuda_check(sim, cudaStreamSynchronize(sim->st), "sync");
    dev_free(sim, tp);
    dev_free(sim, tv);
    dev_free(sim, ti);
    if (rc != BBMD_OK) return rc;
    return read_status(sim);
}

bbmd_status bbmd_set_state(bbmd_sim* sim, const double* pos, const double* vel,
                           const int32_t* image) {
    if (!sim || !pos || !vel) return BBMD_ERR_ARG;
    DeviceGuard dg(sim->device);
    finish_velocities(sim);
    const int64_t n = sim->d.n;
    double* tp = (double*)dev_alloc(sim, 3 * n * 8);
    double* tv = (double*)dev_alloc(sim, 3 * n * 8);
    int32_t* ti = image ? (int32_t*)dev_alloc(sim, 3 * n * 4) : nullptr;
    bbmd_status rc = BBMD_OK;
    if (!tp || !tv || (image && !ti)) rc = fail(sim, BBMD_ERR_OOM, "set_state");
    if (rc == BBMD_OK)
        rc = cuda_check(sim, cudaMemcpyAsync(tp, pos, 3 * n * 8, cudaMemcpyHostToDevice, sim->st), "H2D");
    if (rc == BBMD_OK)
        rc = cuda_check(sim, cudaMemcpyAsync(tv, vel, 3 * n * 8, cudaMemcpyHostToDevice, sim->st), "H2D");
    if (rc == BBMD_OK && image)
        rc = cuda_check(sim, cudaMemcpyAsync(ti, image, 3 * n * 4, cudaMemcpyHostToDevice, sim->st), "H2D");
    // the uploaded values are checked on the device (one pass over them at HBM speed, not
    // a serial host scan) before anything of the state is replaced
    if (rc == BBMD_OK) {
        int bad = 0;
        rc = cuda_check(sim, cudaMemsetAsync(&sim->d.sc->bad_input, 0, sizeof(int), sim->st), "memset");
        if (rc == BBMD_OK) {
            launch_check_finite(sim->d, sim->st, tp, 3 * n);
            launch_check_finite(sim->d, sim->st, tv, 3 * n);
            rc = cuda_check(sim, cudaMemcpyAsync(&bad, &sim->d.sc->bad_input, sizeof(int),
                                                 cudaMemcpyDeviceToHost, sim->st), "D2H");
        }
        if (rc == BBMD_OK) rc = cuda_check(sim, cudaStreamSynchronize(sim->st), "sync");
        if (rc == BBMD_OK && bad) rc = fail(sim, BBMD_ERR_ARG, "non-finite positions or velocities");
    }
    if (rc == BBMD_OK) {
        launch_pack_state(sim->d, sim->st, tp, tv, ti, true);
        rc = cuda_check(sim, cudaGetLastError(), "pack");
    }
    if (rc == BBMD_OK) rc = rebuild_now(sim);
    if (rc == BBMD_OK) rc = refresh_forces_and_K(sim);
    if (rc == BBMD_OK) rc = cuda_check(sim, cudaStreamSynchronize(sim->st), "sync");
    dev_free(sim, tp);
    dev_free(sim, tv);
    dev_free(sim, ti);
    if (rc != BBMD_OK) return rc;
    return read_status(sim);
}

bbmd_status bbmd_get_forces_ids(bbmd_sim* sim, const int64_t* ids, int64_t m, double* F,
                                double* u) {
    if (!sim || !ids || !F || m < 0) return BBMD_ERR_ARG;
    DeviceGuard dg(sim->device);
    const int64_t n = sim->d.n;
    for (int64_t t = 0; t < m; ++t)
        if (ids[t] < 0 || ids[t] >= n) return fail(sim, BBMD_ERR_ARG, "ids must be in [0, n)");
    if (m == 0) return BBMD_OK;
    launch_force(sim->d, sim->st, u != nullptr, false);
    int32_t* slot_of = (int32_t*)dev_alloc(sim, (size_t)n * 4);
    int64_t* dids = (int64_t*)dev_alloc(sim, (size_t)m * 8);
    double* tf = (double*)dev_alloc(sim, (size_t)m * 24);
    double* tu = u ? (double*)dev_alloc(sim, (size_t)m * 8) : nullptr;
    bbmd_status rc = BBMD_OK;
    if (!slot_of || !dids || !tf || (u && !tu)) rc = fail(sim, BBMD_ERR_OOM, "get_forces_ids");
    if (rc == BBMD_OK)
        rc = cuda_check(sim, cudaMemcpyAsync(dids, ids, (size_t)m * 8, cudaMemcpyHostToDevice, sim->st), "H2D");
    if (rc == BBMD_OK) {
        launch_slot_of(sim->d, sim->st, slot_of);
        launch_forces_of_ids(sim->d, sim->st, slot_of, dids, m, tf, tu);
        rc = cuda_check(sim, cudaGetLastError(), "forces of ids");
    }
    if (rc == BBMD_OK)
        rc = cuda_check(sim, cudaMemcpyAsync(F, tf, (size_t)m * 24, cudaMemcpyDeviceToHost, sim->st), "D2H");
    if (rc == BBMD_OK && u)
        rc = cuda_check(sim, cudaMemcpyAsync(u, tu, (size_t)m * 8, cudaMemcpyDeviceToHost, sim->st), "D2H");
    if (rc == BBMD_OK) rc = cuda_check(sim, cudaStreamSynchronize(sim->st), "sync");
    dev_free(sim, slot_of);
    dev_free(sim, dids);
    dev_free(sim, tf);
    dev_free(sim, tu);
    if (rc != BBMD_OK) return rc;
    return read_status(sim);
}

bbmd_status bbmd_get_forces(bbmd_sim* sim, double* F, double* u) {
    if (!sim || !F) return BBMD_ERR_ARG;
    DeviceGuard dg(sim->device);
    const int64_t n = sim->d.n;
    launch_force(sim->d, sim->st, u != nullptr, false);
    double* tf = (double*)dev_alloc(sim, 3 * n * 8);
    double* tu = u ? (double*)dev_alloc(sim, n * 8) : nullptr;
    bbmd_status rc = BBMD_OK;
    if (!tf || (u && !tu)) rc = fail(sim, BBMD_ERR_OOM, "get_forces");
    if (rc == BBMD_OK) {
        launch_unpack_forces(sim->d, sim->st, tf, tu);
        rc = cuda_check(sim, cudaGetLastError(), "unpack forces");
    }
    if (rc == BBMD_OK)
        rc = cuda_check(sim, cudaMemcpyAsync(F, tf, 3 * n * 8, cudaMemcpyDeviceToHost, sim->st), "D2H");
    if (rc == BBMD_OK && u)
        rc = cuda_check(sim, cudaMemcpyAsync(u, tu, n * 8, cudaMemcpyDeviceToHost, sim->st), "D2H");
    if (rc == BBMD_OK) rc = cuda_check(sim, cudaStreamSynchronize(sim->st), "sync");
    dev_free(sim, tf);
    dev_free(sim, tu);
    if (rc != BBMD_OK) return rc;
    return read_status(sim);
}

bbmd_status bbmd_get_cells(bbmd_sim* sim, int64_t* cell) {
    if (!sim || !cell) return BBMD_ERR_ARG;
    DeviceGuard dg(sim->device);
    const int64_t n = sim->d.n;
    int64_t* tc = (int64_t*)dev_alloc(sim, n * 8);
    if (!tc) return fail(sim, BBMD_ERR_OOM, "get_cells");
    launch_unpack_cells(sim->d, sim->st, tc);
    bbmd_status rc = cuda_check(sim, cudaGetLastError(), "unpack cells");
    if (rc == BBMD_OK)
        rc = cuda_check(sim, cudaMemcpyAsync(cell, tc, n * 8, cudaMemcpyDeviceToHost, sim->st), "D2H");
    if (rc == BBMD_OK) rc = cuda_check(sim, cudaStreamSynchronize(sim->st), "sync");
    dev_free(sim, tc);
    return rc;
}

bbmd_status bbmd_get_neighbors(bbmd_sim* sim, const int64_t* ids, int64_t m, int64_t* offsets,
                               int64_t* nbr, int64_t cap) {
    if (!sim || !offsets) return BBMD_ERR_ARG;
    DeviceGuard dg(sim->device);
    if (sim->d.nbr_mode != BBMD_NBR_VERLET) return fail(sim, BBMD_ERR_STATE, "no stored list in cell mode");
    {
        const bbmd_status g = read_status(sim);  // grows cut lists first
        if (g != BBMD_OK) return g;
    }
    const int64_t n = sim->d.n;
    if (!ids) m = n;
    if (m < 0 || m > n) return fail(sim, BBMD_ERR_ARG, "m");
    int32_t* sel = nullptr;
    if (ids) {
        std::vector<int32_t> slot((size_t)n);
        for (int64_t t = 0; t < m; ++t)
            if (ids[t] < 0 || ids[t] >= n) return fail(sim, BBMD_ERR_ARG, "id out of range");
        int32_t* slot_of = (int32_t*)dev_alloc(sim, n * 4);
        sel = (int32_t*)dev_alloc(sim, (m + 1) * 4);
        if (!slot_of || !sel) {
            dev_free(sim, slot_of);
            dev_free(sim, sel);
            return fail(sim, BBMD_ERR_OOM, "get_neighbors");
        }
        launch_slot_of(sim->d, sim->st, slot_of);
        CK(cudaMemcpyAsync(slot.data(), slot_of, n * 4, cudaMemcpyDeviceToHost, sim->st));
        CK(cudaStreamSynchronize(sim->st));
        std::vector<int32_t> hs((size_t)m + 1);
        for (int64_t t = 0; t < m; ++t) hs[(size_t)t] = slot[(size_t)ids[t]];
        CK(cudaMemcpyAsync(sel, hs.data(), m * 4, cudaMemcpyHostToDevice, sim->st));
        CK(cudaStreamSynchronize(sim->st));
        dev_free(sim, slot_of);
    }
    int64_t* tcnt = (int64_t*)dev_alloc(sim, (m + 1) * 8);
    if (!tcnt) {
        dev_free(sim, sel);
        return fail(sim, BBMD_ERR_OOM, "get_neighbors");
    }
    launch_list_counts(sim->d, sim->st, sel, m, tcnt);
    std::vector<int64_t> cnt((size_t)m + 1);
    bbmd_status rc = cuda_check(sim, cudaGetLastError(), "list counts");
    if (rc == BBMD_OK && m > 0)
        rc = cuda_check(sim, cudaMemcpyAsync(cnt.data(), tcnt, m * 8, cudaMemcpyDeviceToHost, sim->st), "D2H");
    if (rc == BBMD_OK) rc = cuda_check(sim, cudaStreamSynchronize(sim->st), "sync");
    if (rc == BBMD_OK) {
        offsets[0] = 0;
        for (int64_t t = 0; t < m; ++t) offsets[t + 1] = offsets[t] + cnt[(size_t)t];
    }
    if (rc == BBMD_OK && nbr) {
        if (cap < offsets[m]) {
            rc = fail(sim, BBMD_ERR_ARG, "neighbour buffer too small");
        } else {
            int64_t* tnb = (int64_t*)dev_alloc(sim, (offsets[m] + 1) * 8);
            if (!tnb) rc = fail(sim, BBMD_ERR_OOM, "get_neighbors");
            if (rc == BBMD_OK && m > 0)
                rc = cuda_check(sim, cudaMemcpyAsync(tcnt, offsets, m * 8, cudaMemcpyHostToDevice, sim->st), "H2D");
            if (rc == BBMD_OK) {
                launch_list_ids(sim->d, sim->st, sel, m, tcnt, tnb);
                rc = cuda_check(sim, cudaGetLastError(), "list ids");
            }
            if (rc == BBMD_OK && offsets[m] > 0)
                rc = cuda_check(sim, cudaMemcpyAsync(nbr, tnb, offsets[m] * 8, cudaMemcpyDeviceToHost, sim->st), "D2H");
            if (rc == BBMD_OK) rc = cuda_check(sim, cudaStreamSynchronize(sim->st), "sync");
            dev_free(sim, tnb);
        }
    }
    dev_free(sim, tcnt);
    dev_free(sim, sel);
    if (rc != BBMD_OK) return rc;
    return read_status(sim);
}

bbmd_status bbmd_tune(bbmd_sim* sim) {
    if (!sim) return BBMD_ERR_ARG;
    DeviceGuard dg(sim->device);
    finish_velocities(sim);
    if (sim->shapes.size() < 2) return BBMD_OK;
    // weight of the list build: the rebuilds per step seen since the last tuning (a rebuild
    // about every four steps when fewer than 20 steps were taken)
    DevScalars scl;
    CK(cudaMemcpyAsync(&scl, sim->d.sc, sizeof(scl), cudaMemcpyDeviceToHost, sim->st));
    CK(cudaStreamSynchronize(sim->st));
    float rate = 0.25f;
    const long long dsteps = scl.step - sim->tune_step, dreb = scl.n_rebuilds - sim->tune_rebuilds;
    if (dsteps >= 20) rate = std::min(1.0f, std::max(0.02f, (float)dreb / (float)dsteps));
    sim->tune_step = scl.step;
    sim->tune_rebuilds = scl.n_rebuilds;
    bbmd_status rc = rebuild_now(sim);
    if (rc == BBMD_OK) rc = autotune_shape(sim, rate);
    free_graphs(sim);  // the captured launches carry the previous shape
    if (rc == BBMD_OK) rc = refresh_forces_and_K(sim);
    if (rc != BBMD_OK) return rc;
    return read_status(sim);
}

bbmd_status bbmd_rebuild(bbmd_sim* sim) {
    if (!sim) return BBMD_ERR_ARG;
    DeviceGuard dg(sim->device);
    finish_velocities(sim);
    bbmd_status rc = rebuild_now(sim);
    if (rc != BBMD_OK) return rc;
    launch_force(sim->d, sim->st, false, false);
    LAUNCHED("rebuild forces");
    return read_status(sim);
}

bbmd_status bbmd_get_info(const bbmd_sim* sim, bbmd_info* info) {
    if (!sim || !info) return BBMD_ERR_ARG;
    info->n = sim->d.n;
    info->fix_exponent = sim->d.kexp;
    for (int d = 0; d < 3; ++d) {
        info->nc[d] = sim->d.nc[d];
        info->cell_side_fix[d] = sim->d.D[d];
    }
    info->list_capacity = sim->d.lcap8 * 8;
    info->stencil_capacity = sim->d.smax;
    info->block_z = sim->d.block_z;
    for (int k = 0; k < 4; ++k) {
        info->shape_force_ms[k] = sim->shape_ms[k][0];
        info->shape_list_ms[k] = sim->shape_ms[k][1];
    }
    info->device_bytes = sim->bytes;
    return BBMD_OK;
}

const char* bbmd_last_error(const bbmd_sim* sim) { return sim ? sim->err.c_str() : ""; }

}  // extern "C"

// ------------------------------------------------------------------- replica batches ----

struct bbmd_batch {
    std::vector<bbmd_sim*> rep;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // [thermostatted]
    std::vector<int> gen[2];         // replicas' graph generations at capture
    std::vector<void*> dev;          // device tables of the batch launches
    int branches = 8;                // graph branches, each a group of replicas
    std::vector<std::function<void()>> pending;  // per branch: its launches (during capture)
    std::vector<cudaStream_t> side;  // capture streams of the branches
    std::vector<cudaEvent_t> ev;     // fork + joins
    std::string err;
    int device = 0;                  // CUDA device of every replica (current at creation)
    int mode = BBMD_BATCH_AUTO;      // step path requested (bbmd_batch_set_mode)
    // persistent step: launch tables, barrier word, grid, staged capacity, generations
    PersistentStep pst = {};
    std::vector<void*> pdev;         // device tables of the persistent step
    int32_t* pctl = nullptr;         // its control words: queue head, finished counts, abort
    size_t pctl_bytes = 0;           // bytes of head + finished counts (cleared every launch)
    int pgrid = 0, psmax = 0;
    std::vector<int> pgen;           // replicas' graph generations at the table upload
    uint64_t wait_ns = 1000000000ull;  // dependency-wait limit of the persistent step
};

namespace {

constexpr int64_t kPersistSteps = 1024;  // steps per launch of the persistent step

bbmd_status batch_fail(bbmd_batch* b, bbmd_status code, const std::string& msg) {
    if (b) b->err = msg;
    return code;
}

void batch_free_graphs(bbmd_batch* b) {
    for (auto& g : b->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

void batch_free_tables(bbmd_batch* b) {
    for (void* p : b->dev) cudaFree(p);
    b->dev.clear();
}

void batch_free_persistent(bbmd_batch* b) {
    for (void* p : b->pdev) cudaFree(p);
    b->pdev.clear();
    b->pgen.clear();
    b->pctl = nullptr;
}

// The persistent step applies when every replica is mixed precision with the block shape
// of the persistent kernel and the device runs cooperative launches.
bool persistent_eligible(const bbmd_batch* b) {
    int coop = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, b->device) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (!coop) return false;
    for (const bbmd_sim* s : b->rep)
        if (s->d.precision != BBMD_PREC_MIXED || s->d.block_z != kPersistZ) return false;
    return true;
}

// Upload systems and CTA offsets for one set of replicas; returns the ManySims view and
// the total CTA count, or false on a CUDA error.
bool upload_many(bbmd_batch* b, const std::vector<const DevSim*>& sims,
                 const std::vector<int32_t>& ctas, ManySims& m, int& total) {
    const size_t nr = sims.size();
    std::vector<DevSim> hs(nr);
    std::vector<int32_t> first(nr + 1, 0);
    for (size_t r = 0; r < nr; ++r) {
        hs[r] = *sims[r];
        first[r + 1] = first[r] + ctas[r];
    }
    void* ds = nullptr;
    void* df = nullptr;
    if (cudaMalloc(&ds, nr * sizeof(DevSim)) != cudaSuccess) return false;
    b->dev.push_back(ds);
    if (cudaMalloc(&df, (nr + 1) * sizeof(int32_t)) != cudaSuccess) return false;
    b->dev.push_back(df);
    if (cudaMemcpy(ds, hs.data(), nr * sizeof(DevSim), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(df, first.data(), (nr + 1) * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess)
        return false;
    m.sims = (const DevSim*)ds;
    m.first = (const int32_t*)df;
    m.nrep = (int32_t)nr;
    total = first[nr];
    return true;
}


// Tables of the persistent step for the current replicas: their DevSims, the work items
// of one step in phase-major order, the items per replica and phase, each phase's
// predecessor, the control words (queue head and finished counts, then the abort flag),
// and the grid: every SM's resident CTAs.
bbmd_status build_persistent(bbmd_batch* b) {
    cudaStreamSynchronize(b->st);
    batch_free_persistent(b);
    const int nr = (int)b->rep.size();
    // Per-particle and per-cell phases take one item per 2048 particles of a replica (the
    // device copies of the replicas' DevSims carry that count as grid_part): an item then
    // outweighs its set-up, and no result of those phases depends on how the particles
    // are split.  Forces and list builds keep the replica's own CTA counts (the
    // kinetic-energy partials are summed over grid_cell).
    std::vector<DevSim> copies((size_t)nr);
    std::vector<int32_t> need((size_t)nr * kPhases, 0), dep((size_t)nr * kPhases, -1);
    int smax = 0;
    for (int r = 0; r < nr; ++r) {
        DevSim& c = copies[(size_t)r];
        c = b->rep[(size_t)r]->d;
        c.grid_part = (int32_t)std::max<int64_t>(1, (c.n + 2047) / 2048);
        smax = std::max(smax, (int)c.smax);
        int32_t* nd = &need[(size_t)r * kPhases];
        for (int ph = 0; ph < kPhases; ++ph) nd[ph] = c.grid_part;
        nd[kPhScan] = 1;
        nd[kPhList] = c.nbr_mode == BBMD_NBR_VERLET ? c.grid_list : 0;
        nd[kPhForce] = c.grid_cell;
        nd[kPhFinalize] = 1;
        int last = -1;
        for (int ph = 0; ph < kPhases; ++ph) {
            dep[(size_t)r * kPhases + ph] = last;
            if (nd[ph] > 0) last = ph;
        }
    }
    std::vector<int4> items;
    for (int ph = 0; ph < kPhases; ++ph)
        for (int r = 0; r < nr; ++r) {
            const int c = need[(size_t)r * kPhases + ph];
            for (int k = 0; k < c; ++k) items.push_back(make_int4(ph, r, k, c));
        }
    auto upload = [&](const void* host, size_t bytes) -> void* {
        void* d = nullptr;
        if (cudaMalloc(&d, bytes) != cudaSuccess) return nullptr;
        b->pdev.push_back(d);
        if (host && cudaMemcpy(d, host, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return nullptr;
        return d;
    };
    PersistentStep& a = b->pst;
    a.sims = (const DevSim*)upload(copies.data(), copies.size() * sizeof(DevSim));
    a.items = (const int4*)upload(items.data(), items.size() * sizeof(int4));
    a.need = (const int32_t*)upload(need.data(), need.size() * sizeof(int32_t));
    a.dep = (const int32_t*)upload(dep.data(), dep.size() * sizeof(int32_t));
    // control words: head, done[nrep][kPhases], abort
    b->pctl_bytes = (1 + need.size()) * sizeof(int32_t);
    int32_t* ctl = (int32_t*)upload(nullptr, b->pctl_bytes + sizeof(int32_t));
    if (!a.sims || !a.items || !a.need || !a.dep || !ctl) {
        cudaGetLastError();
        batch_free_persistent(b);
        return batch_fail(b, BBMD_ERR_OOM, "persistent step tables");
    }
    a.head = (uint32_t*)ctl;
    a.done = ctl + 1;
    a.abort = ctl + 1 + need.size();
    a.nrep = nr;
    a.nitems = (int32_t)items.size();
    b->pctl = ctl;
    if (!BBMD_PERSIST_NS::prepare_persistent()) {
        cudaGetLastError();
        return batch_fail(b, BBMD_ERR_CUDA, "persistent step shared memory");
    }
    const int per_sm = BBMD_PERSIST_NS::persistent_blocks_per_sm(smax);
    if (per_sm < 1) return batch_fail(b, BBMD_ERR_CUDA, "persistent step does not fit an SM");
    b->pgrid = per_sm * b->rep[0]->nsm;
    b->psmax = smax;
    b->pgen.resize((size_t)nr);
    for (int r = 0; r < nr; ++r) b->pgen[(size_t)r] = b->rep[(size_t)r]->graph_gen;
    return BBMD_OK;
}

// Launches of one step for a group of replicas: one launch per phase for the whole group
// (integrate, the gated sort chain, the gated list build and the forces -- one launch per
// block shape in use -- and finalize).
bool capture_group(bbmd_batch* b, const std::vector<size_t>& idx, int nh, cudaStream_t st) {
    const size_t nr = idx.size();
    const DevSim& D0 = b->rep[idx[0]]->d;
    const bool fp64 = D0.precision == BBMD_PREC_FP64;
    const bool cell = D0.nbr_mode != BBMD_NBR_VERLET;
    const bool fshift = D0.pt.shift == BBMD_SHIFT_FORCE;
    std::vector<const DevSim*> all(nr);
    std::vector<int32_t> c_part(nr), c_scan(nr), c_one(nr, 1);
    for (size_t r = 0; r < nr; ++r) {
        all[r] = &b->rep[idx[r]]->d;
        c_part[r] = all[r]->grid_part;
        c_scan[r] = scan_grid(*all[r]);
    }
    ManySims part, scan, one;
    int t_part = 0, t_scan = 0, t_one = 0;
    if (!(upload_many(b, all, c_part, part, t_part) && upload_many(b, all, c_scan, scan, t_scan) &&
          upload_many(b, all, c_one, one, t_one)))
        return false;
    struct Group {
        int bz;
        ManySims force, list;
        int t_force = 0, t_list = 0, smax = 0;
    };
    std::vector<Group> groups;
    for (int bz : kShapes) {
        std::vector<const DevSim*> gs;
        std::vector<int32_t> c_force, c_list;
        int smax = 0;
        for (size_t r = 0; r < nr; ++r)
            if (all[r]->block_z == bz) {
                gs.push_back(all[r]);
                c_force.push_back(all[r]->grid_cell);
                c_list.push_back(all[r]->grid_list);
                smax = std::max(smax, (int)all[r]->smax);
            }
        if (gs.empty()) continue;
        Group g;
        g.bz = bz;
        g.smax = smax;
        if (!(upload_many(b, gs, c_force, g.force, g.t_force) &&
              upload_many(b, gs, c_list, g.list, g.t_list)))
            return false;
        groups.push_back(g);
    }
    // the tables are uploaded (synchronous copies) now; the launches run in the capture
    b->pending.push_back([=]() {
        launch_integrate_many(part, t_part, fp64, st);
        launch_check_many(part, t_part, st);
        launch_rebuild_chain_many(part, scan, one, t_part, t_scan, (int)nr, st);
        for (const Group& g : groups) {
            if (cell) continue;
            switch (g.bz) {
                case 1: z1::launch_list_build_many(g.list, g.t_list, g.smax, st); break;
                case 2: z2::launch_list_build_many(g.list, g.t_list, g.smax, st); break;
                case 4: z4::launch_list_build_many(g.list, g.t_list, g.smax, st); break;
                default: z8::launch_list_build_many(g.list, g.t_list, g.smax, st); break;
            }
        }
        for (const Group& g : groups) {
            switch (g.bz) {
                case 1: z1::launch_force_many(g.force, g.t_force, fp64, cell, nh != 0, fshift, g.smax, st); break;
                case 2: z2::launch_force_many(g.force, g.t_force, fp64, cell, nh != 0, fshift, g.smax, st); break;
                case 4: z4::launch_force_many(g.force, g.t_force, fp64, cell, nh != 0, fshift, g.smax, st); break;
                default: z8::launch_force_many(g.force, g.t_force, fp64, cell, nh != 0, fshift, g.smax, st); break;
            }
        }
        launch_finalize_many(one, (int)nr, nh != 0, st);
    });
    return true;
}

// One graph for one step of every replica: the replicas are split into `branches` groups
// of about equal particle count (largest first, each to the lightest group); the graph
// forks into one branch per group, each branch running its group's phase launches, and
// joins.  Groups overlap one another's phases; within a group one launch covers all its
// replicas.
bbmd_status build_batch_graph(bbmd_batch* b, int nh) {
    cudaStreamSynchronize(b->st);
    batch_free_graphs(b);
    batch_free_tables(b);
    b->pending.clear();
    const size_t nr = b->rep.size();
    const size_t nb = std::max<size_t>(1, std::min<size_t>((size_t)b->branches, nr));
    std::vector<size_t> order(nr);
    for (size_t r = 0; r < nr; ++r) order[r] = r;
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t x, size_t y) { return b->rep[x]->d.n > b->rep[y]->d.n; });
    std::vector<std::vector<size_t>> grp(nb);
    std::vector<int64_t> load(nb, 0);
    for (size_t r : order) {
        size_t k = 0;
        for (size_t q = 1; q < nb; ++q)
            if (load[q] < load[k]) k = q;
        grp[k].push_back(r);
        load[k] += b->rep[r]->d.n;
    }
    for (auto& g : grp) std::sort(g.begin(), g.end());
    while (b->side.size() < nb) {
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
            return batch_fail(b, BBMD_ERR_CUDA, "batch streams");
        b->side.push_back(st);
    }
    while (b->ev.size() < nb + 1) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return batch_fail(b, BBMD_ERR_CUDA, "batch events");
        b->ev.push_back(e);
    }
    for (size_t k = 0; k < nb; ++k)
        if (!capture_group(b, grp[k], nh, b->side[k])) {
            cudaGetLastError();
            return batch_fail(b, BBMD_ERR_OOM, "batch launch tables");
        }
    cudaError_t e = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return batch_fail(b, BBMD_ERR_CUDA, cudaGetErrorString(e));
    cudaEventRecord(b->ev[0], b->st);
    for (size_t k = 0; k < nb; ++k) {
        cudaStreamWaitEvent(b->side[k], b->ev[0], 0);
        b->pending[k]();
        cudaEventRecord(b->ev[k + 1], b->side[k]);
        cudaStreamWaitEvent(b->st, b->ev[k + 1], 0);
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->st, &g);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph[nh], g, 0);
    if (g) cudaGraphDestroy(g);
    b->pending.clear();
    if (e != cudaSuccess) {
        cudaGetLastError();
        b->graph[nh] = nullptr;
        return batch_fail(b, BBMD_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
    }
    for (int k = 0; k < 2; ++k) b->gen[k].clear();
    b->gen[nh].resize(nr);
    for (size_t r = 0; r < nr; ++r) b->gen[nh][r] = b->rep[r]->graph_gen;
    return BBMD_OK;
}

}  // namespace

extern "C" {

void bbmd_destroy_batch(bbmd_batch* b) {
    if (!b) return;
    DeviceGuard dg(b->device);
    if (b->st) cudaStreamSynchronize(b->st);
    batch_free_graphs(b);
    batch_free_tables(b);
    batch_free_persistent(b);
    for (bbmd_sim* s : b->rep) bbmd_destroy(s);
    for (cudaStream_t s : b->side) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    if (b->own_stream) cudaStreamDestroy(b->st);
    delete b;
}

bbmd_status bbmd_create_batch(const bbmd_params* params, int32_t n_rep, const int64_t* n,
                              const double* box, const uint8_t* const* species,
                              const double* const* pos, const double* const* vel,
                              const double* T0, uint64_t seed, void* stream,
                              const bbmd_alloc* alloc, bbmd_batch** out) {
    if (!out) return BBMD_ERR_ARG;
    *out = nullptr;
    if (!params || n_rep < 1 || n_rep > 65536 || !n || !box || !species || !T0)
        return BBMD_ERR_ARG;
    bbmd_batch* b = new bbmd_batch();
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return BBMD_ERR_CUDA;
    }
    b->st = (cudaStream_t)stream;
    if (!b->st) {
        if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return BBMD_ERR_CUDA;
        }
        b->own_stream = true;
    }
    bbmd_status rc = BBMD_OK;
    // the replicas of a batch share one block shape; 0 selects the shape of the persistent
    // step
    bbmd_params P = *params;
    if (P.block_z == 0) P.block_z = kPersistZ;
    for (int32_t r = 0; r < n_rep && rc == BBMD_OK; ++r) {
        bbmd_sim* s = nullptr;
        rc = bbmd_create(&P, n[r], box + 3 * (size_t)r, species[r], pos ? pos[r] : nullptr,
                         vel ? vel[r] : nullptr, T0[r], seed + (uint64_t)r, b->st, alloc, &s);
        if (rc == BBMD_OK) b->rep.push_back(s);
    }
    if (rc != BBMD_OK) {
        bbmd_destroy_batch(b);
        return rc;
    }
    *out = b;
    return BBMD_OK;
}

bbmd_status bbmd_step_batch(bbmd_batch* b, int64_t nsteps, double dt, const bbmd_thermostat* th) {
    if (!b) return BBMD_ERR_ARG;
    DeviceGuard dg(b->device);
    if (nsteps < 0 || nsteps > 0x7fffffff || !(dt > 0.0) || !(dt < 1.0))
        return batch_fail(b, BBMD_ERR_ARG, "nsteps in [0, 2^31) and dt in (0, 1) required");
    int nh = 0;
    if (th) {
        nh = th[0].kind == BBMD_THERMO_NH;
        for (size_t r = 0; r < b->rep.size(); ++r) {
            if (th[r].kind != th[0].kind)
                return batch_fail(b, BBMD_ERR_ARG, "all replicas need the same thermostat kind");
            if (th[r].kind != BBMD_THERMO_NVE && th[r].kind != BBMD_THERMO_NH)
                return batch_fail(b, BBMD_ERR_ARG, "thermostat kind");
            if (nh && !(th[r].T_start > 0.0 && th[r].T_end > 0.0 && th[r].tau > 0.0))
                return batch_fail(b, BBMD_ERR_ARG, "Nose-Hoover needs T_start, T_end, tau > 0");
        }
    }
    if (nsteps == 0) return BBMD_OK;
    const bool persistent = b->mode != BBMD_BATCH_GRAPH && persistent_eligible(b);
    if (b->mode == BBMD_BATCH_PERSISTENT && !persistent)
        return batch_fail(b, BBMD_ERR_STATE,
                          "the persistent step needs mixed precision, the batch block shape and "
                          "cooperative launch");
    if (persistent) {
        bool pstale = b->pgen.size() != b->rep.size();
        for (size_t r = 0; !pstale && r < b->rep.size(); ++r)
            pstale = b->pgen[r] != b->rep[r]->graph_gen;
        if (pstale) {
            bbmd_status rc = build_persistent(b);
            if (rc != BBMD_OK) return rc;
        }
        const bool fshift = b->rep[0]->d.pt.shift == BBMD_SHIFT_FORCE;
        for (size_t r = 0; r < b->rep.size(); ++r)
            begin_call(b->rep[r], nsteps, dt, nh ? &th[r] : nullptr);
        // the abort flag is cleared once per call, the queue head and the finished counts
        // before every launch; a launch runs up to kPersistSteps steps (the queue counts
        // items of one launch in 32 bits)
        cudaError_t e0 = cudaMemsetAsync(b->pst.abort, 0, sizeof(int32_t), b->st);
        if (e0 != cudaSuccess) return batch_fail(b, BBMD_ERR_CUDA, cudaGetErrorString(e0));
        const int64_t per_launch =
            std::max<int64_t>(1, std::min<int64_t>(kPersistSteps, 0x7fffffff / std::max(1, b->pst.nitems)));
        for (int64_t k = 0; k < nsteps; k += per_launch) {
            PersistentStep a = b->pst;
            a.nsteps = (int32_t)std::min<int64_t>(per_launch, nsteps - k);
            a.wait_ns = b->wait_ns;
            cudaError_t e = cudaMemsetAsync(b->pctl, 0, b->pctl_bytes, b->st);
            if (e == cudaSuccess)
                e = BBMD_PERSIST_NS::launch_persistent_step(a, b->pgrid, b->psmax, nh != 0, fshift, b->st);
            if (e != cudaSuccess) return batch_fail(b, BBMD_ERR_CUDA, cudaGetErrorString(e));
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return batch_fail(b, BBMD_ERR_CUDA, cudaGetErrorString(e));
        return BBMD_OK;
    }
    bool stale = !b->graph[nh] || b->gen[nh].size() != b->rep.size();
    for (size_t r = 0; !stale && r < b->rep.size(); ++r)
        stale = b->gen[nh][r] != b->rep[r]->graph_gen;
    if (stale) {
        bbmd_status rc = build_batch_graph(b, nh);
        if (rc != BBMD_OK) return rc;
    }
    for (size_t r = 0; r < b->rep.size(); ++r)
        begin_call(b->rep[r], nsteps, dt, nh ? &th[r] : nullptr);
    for (int64_t k = 0; k < nsteps; ++k) {
        cudaError_t e = cudaGraphLaunch(b->graph[nh], b->st);
        if (e != cudaSuccess) return batch_fail(b, BBMD_ERR_CUDA, cudaGetErrorString(e));
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return batch_fail(b, BBMD_ERR_CUDA, cudaGetErrorString(e));
    return BBMD_OK;
}

bbmd_sim* bbmd_batch_replica(bbmd_batch* b, int32_t r) {
    if (!b || r < 0 || (size_t)r >= b->rep.size()) return nullptr;
    return b->rep[(size_t)r];
}

int32_t bbmd_batch_size(const bbmd_batch* b) { return b ? (int32_t)b->rep.size() : 0; }

bbmd_status bbmd_batch_set_mode(bbmd_batch* b, int32_t mode) {
    if (!b || mode < BBMD_BATCH_AUTO || mode > BBMD_BATCH_PERSISTENT) return BBMD_ERR_ARG;
    b->mode = mode;
    return BBMD_OK;
}

int32_t bbmd_batch_uses_persistent(const bbmd_batch* b) {
    if (!b) return 0;
    return b->mode != BBMD_BATCH_GRAPH && persistent_eligible(b) ? 1 : 0;
}

bbmd_status bbmd_batch_set_wait_limit(bbmd_batch* b, uint64_t ns) {
    if (!b || ns == 0) return BBMD_ERR_ARG;
    b->wait_ns = ns;
    return BBMD_OK;
}

bbmd_status bbmd_batch_set_branches(bbmd_batch* b, int32_t branches) {
    if (!b || branches < 1) return BBMD_ERR_ARG;
    b->branches = branches;
    for (auto& g : b->gen) g.clear();  // re-captured at the next step
    return BBMD_OK;
}

const char* bbmd_batch_last_error(const bbmd_batch* b) { return b ? b->err.c_str() : ""; }

}  // extern "C"

// ----------------------------------------------------- g(r) without device allocation ----
// Who cannot allocate: a system sized to fill HBM has no room left for the g(r) buffers that
// bbmd_observe grows on first use; cudaMalloc / cudaFree (and a caching allocator returning
// memory to the driver) can synchronise the whole device, which would stall the stepping
// stream of a monitoring loop that samples g(r) between steps; code running inside an
// allocator callback must not call back into the allocator.  This variant takes its scratch
// from one fixed array compiled into the library instead.
static __device__ __align__(256) int32_t noalloc_scratch[BBMD_NOALLOC_GR_SCRATCH_INTS];
static __device__ __align__(256) unsigned long long noalloc_counts[4 * BBMD_NOALLOC_GR_MAX_BINS];

namespace {

constexpr int64_t kNoAllocInts = BBMD_NOALLOC_GR_SCRATCH_INTS;
constexpr int kNoAllocBins = BBMD_NOALLOC_GR_MAX_BINS;
constexpr int kNoAllocDevices = 64;

struct NoAllocSlot {
    int32_t* scratch;
    unsigned long long* counts;
};
NoAllocSlot noalloc_slot[kNoAllocDevices];  // per device, filled by the first call there

bbmd_status noalloc_setup(bbmd_sim* sim, int dev) {
    NoAllocSlot& sl = noalloc_slot[dev];
    if (sl.scratch && sl.counts) return BBMD_OK;
    void* a = nullptr;
    void* b = nullptr;
    CK(cudaGetSymbolAddress(&a, noalloc_scratch));
    CK(cudaGetSymbolAddress(&b, noalloc_counts));
    sl.scratch = (int32_t*)a;
    sl.counts = (unsigned long long*)b;
    return BBMD_OK;
}

}  // namespace

extern "C" bbmd_status bbmd_gr_counts_noalloc(bbmd_sim* sim, int32_t nbins, double rmax,
                                              uint64_t* counts) {
    if (!sim || !counts) return BBMD_ERR_ARG;
    DeviceGuard dg(sim->device);
    if (nbins <= 0) nbins = 500;
    if (!(rmax > 0.0)) rmax = 5.0;
    if (nbins > kNoAllocBins) return fail(sim, BBMD_ERR_ARG, "nbins <= 4096");
    const DevSim& D = sim->d;
    // the scratch the coarse-grid path of launch_gr will ask for (same rule as launch_gr)
    bool cells = true;
    int64_t ncg = 1;
    for (int d = 0; d < 3; ++d) {
        double L = std::ldexp((double)D.Lfix[d], -D.kexp);
        int m = (int)std::floor(L / rmax);
        if (m < 3) cells = false;
        ncg *= m < 1 ? 1 : m;
    }
    const int64_t need = cells ? 2 * D.n + 3 * (ncg + 1) : 0;
    if (need > kNoAllocInts)
        return fail(sim, BBMD_ERR_ARG,
                    "g(r) without allocation: the coarse-grid search needs " +
                        std::to_string(need) + " int32 scratch entries, the fixed array holds " +
                        std::to_string(kNoAllocInts) + " (use bbmd_observe)");
    const int dev = sim->device;
    if (dev < 0 || dev >= kNoAllocDevices) return fail(sim, BBMD_ERR_ARG, "device ordinal >= 64");
    bbmd_status rc = noalloc_setup(sim, dev);
    if (rc != BBMD_OK) return rc;
    const NoAllocSlot& sl = noalloc_slot[dev];
    if (launch_gr(D, sim->st, nbins, rmax, sl.counts, sl.scratch, nullptr, kNoAllocInts) != 0)
        return fail(sim, BBMD_ERR_ARG, "g(r) without allocation: fixed scratch too small");
    LAUNCHED("gr_counts_noalloc");
    CK(cudaMemcpyAsync(counts, sl.counts, sizeof(unsigned long long) * 4 * (size_t)nbins,
                       cudaMemcpyDeviceToHost, sim->st));
    CK(cudaStreamSynchronize(sim->st));
    return read_status(sim);
}
