// Pair forces of the truncated Lennard-Jones / soft-sphere mixture (Sec. 2.1, Eqs. lj0,
// sc0, mod0) over the cell stencil (Sec. 2.2), and the Verlet-list build.
//
// Work unit: one CTA of 8 warps per 2x2x2 block of cells; warp w owns one cell of the block
// (its "tile": up to 32 particles at a time, larger cells in chunks of 32).  The CTA stages
// the 4x4x4 cells around the block -- the union of the eight 27-cell stencils -- into
// shared memory as float4 {x, y, z, species} in one frame (the block's centre).  The raw
// frame-relative records of each cell arrive by one TMA bulk copy per cell (cells are
// contiguous after the counting sort); the exact frame offsets are then added in shared
// memory.  Each lane owns one particle i and accumulates its force in registers: a full
// list, one writer per i, no atomics (the paper applies Newton's third law to halve the
// pair work on a CPU; here every pair is visited from both sides so that each force has
// a single owner and a fixed summation order).
//
// The Verlet list stores, per particle, uint16 offsets into the block's staged array,
// laid out as [kb][npad][8] so a warp reads 8 entries per lane with one coalesced 16-byte
// load.  Padding entries point to a sentinel far outside every cutoff.
//
// Mixed precision: distances and forces in FP32 from block-frame coordinates.  A pair is
// taken as interacting when its FP32 r^2 is below rc^2 (1 - 1e-5); a pair within that
// relative band of the cutoff is decided by the exact FP64 rule in a rare fix-up after
// each batch of 8 pairs, so the interacting set equals the FP64 definition.
//
// This file is compiled once per block shape, code BBMD_BLOCK_Z = 1, 2 or 4 (2 x 2 x Z
// cells) or 8 (4 x 4 x 2 cells), into namespace bbmd::z<BBMD_BLOCK_Z>; the handle picks one
// shape at creation.
#include "bbmd_internal.cuh"

#ifndef BBMD_BLOCK_Z
#error "k_force.cu is compiled once per block shape: define BBMD_BLOCK_Z (code 1, 2, 4 or 8)"
#endif
// warps per CTA and resident CTAs per SM targeted by the force and list kernels, per shape
#if BBMD_BLOCK_Z == 1
#define BBMD_SHAPE_WARPS 4
#define BBMD_SHAPE_FORCE_MIN 6
#define BBMD_SHAPE_LIST_MIN 6
#elif BBMD_BLOCK_Z == 2
#define BBMD_SHAPE_WARPS 8
#define BBMD_SHAPE_FORCE_MIN 3
#define BBMD_SHAPE_LIST_MIN 3
#elif BBMD_BLOCK_Z == 4
#define BBMD_SHAPE_WARPS 8
#define BBMD_SHAPE_FORCE_MIN 2
#define BBMD_SHAPE_LIST_MIN 3
#elif BBMD_BLOCK_Z == 8
#define BBMD_SHAPE_WARPS 8
#define BBMD_SHAPE_FORCE_MIN 2
#define BBMD_SHAPE_LIST_MIN 2
#else
#error "BBMD_BLOCK_Z must be 1, 2, 4 or 8"
#endif
#ifndef BBMD_BLOCK_WARPS
#define BBMD_BLOCK_WARPS BBMD_SHAPE_WARPS
#endif
#ifndef BBMD_FORCE_MIN_BLOCKS
#define BBMD_FORCE_MIN_BLOCKS BBMD_SHAPE_FORCE_MIN
#endif
// the stencil (cell-mode) force kernel of a 2 x 2 x 4 block fits three CTAs per SM in
// shared memory; bounded to them it compiles to 80 registers
#ifndef BBMD_CELL_MIN_BLOCKS
#define BBMD_CELL_MIN_BLOCKS (BBMD_BLOCK_Z == 4 ? 3 : BBMD_FORCE_MIN_BLOCKS)
#endif
#ifndef BBMD_LIST_MIN_BLOCKS
#define BBMD_LIST_MIN_BLOCKS BBMD_SHAPE_LIST_MIN
#endif
#define BBMD_CAT2(a, b) a##b
#define BBMD_CAT(a, b) BBMD_CAT2(a, b)

namespace bbmd {
namespace BBMD_CAT(z, BBMD_BLOCK_Z) {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr float kFar = 1.0e15f;
constexpr int kBlockXY = block_xy_of(BBMD_BLOCK_Z);  // cells of a block along x and y
constexpr int kBlockZ = block_zc_of(BBMD_BLOCK_Z);   // cells of a block along z
constexpr int kRXY = kBlockXY + 2;                   // region cells along x and y
constexpr int kBW = BBMD_BLOCK_WARPS;                // warps per CTA
constexpr int kCells = block_cells_of(BBMD_BLOCK_Z);   // cells per block
constexpr int kRegion = region_cells_of(BBMD_BLOCK_Z);  // cells staged per block
static_assert(kRegion <= kBW * 32, "one thread per staged region cell");
#ifndef BBMD_LIST_AHEAD
#define BBMD_LIST_AHEAD 2
#endif
constexpr int kListAhead = BBMD_LIST_AHEAD;  // list rows in flight ahead of the pair loop
#ifndef BBMD_LIST_PREFETCH
#define BBMD_LIST_PREFETCH 4
#endif
// list rows prefetched into L2 this many rows ahead of the pair loop (0: none), so that
// the register loads two rows ahead find them in L2 rather than in DRAM
constexpr int kListPrefetch = BBMD_LIST_PREFETCH;

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// The region of cells staged for one block: (X + 2) x (Y + 2) x (Z + 2) cells, index
// q = (z * (Y + 2) + y) * (X + 2) + x.
struct Region {
    int off[kRegion + 1];      // prefix of staged counts (clamped to smax); off[kRegion] = total
    int start[kRegion];        // first particle of each region cell
    int cnt[kRegion];          // particles of each region cell
    float hi[kRegion][3];      // frame offset of each cell (FP32 rounding of the exact value)
    float lo[kRegion][3];      // exact residual of that rounding (non-zero across the seam)
    long long fr[kRegion][3];  // FP64 form: frame point + seam image of each cell
    int nstaged;
};

// ------------------------------------------------ TMA bulk copies and mbarriers ----

__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)),
                 "r"(bytes)
                 : "memory");
}

// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) global -> shared,
// completion counted on the mbarrier.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(mbar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the current phase with an iteration limit.  On expiry raise ST_TIMEOUT, wait
// once more (again bounded) for the copies still in flight, and return false.
constexpr int kWaitLimit = 1 << 18;

__device__ __forceinline__ bool mbar_wait_bounded(const DevSim& s, uint64_t* mbar, uint32_t parity) {
    for (int it = 0; it < kWaitLimit; ++it)
        if (mbar_try_wait(mbar, parity)) return true;
    set_status(s, ST_TIMEOUT);
    for (int it = 0; it < kWaitLimit; ++it)
        if (mbar_try_wait(mbar, parity)) break;
    return false;
}

// ------------------------------------------------------------------ blocks ----

struct BlockPos {
    int a0[3];  // first cell of the block per axis
};

__device__ __forceinline__ BlockPos block_pos(const DevSim& s, int64_t blk) {
    const int nbx = (s.nc[0] + kBlockXY - 1) / kBlockXY, nby = (s.nc[1] + kBlockXY - 1) / kBlockXY;
    BlockPos b;
    b.a0[0] = (int)(blk % nbx) * kBlockXY;
    b.a0[1] = (int)((blk / nbx) % nby) * kBlockXY;
    b.a0[2] = (int)(blk / ((int64_t)nbx * nby)) * kBlockZ;
    return b;
}

// Describe the region of block b (threads 0..kRegion-1 take one region cell each): counts,
// frame offsets relative to the block frame, prefix.
__device__ void region_info(const DevSim& s, const BlockPos& b, Region& R) {
    __shared__ int wtot[(kRegion + 31) / 32];
    const int tid = threadIdx.x, lane = tid & 31;
    int cnt = 0;
    if (tid < kRegion) {
        const int r[3] = {tid % kRXY, (tid / kRXY) % kRXY, tid / (kRXY * kRXY)};
        int a[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            int aa = b.a0[d] - 1 + r[d];
            long long wrap = 0;
            if (aa < 0) {
                aa += s.nc[d];
                wrap = -s.Lfix[d];
            } else if (aa >= s.nc[d]) {
                aa -= s.nc[d];
                wrap = s.Lfix[d];
            }
            a[d] = aa;
            // block frame: the cell boundary at the middle of the block (along z, the centre
            // of the cell when the block is one cell high)
            const long long fb = d < 2 ? (long long)(b.a0[d] + kBlockXY / 2) * s.D[d]
                                 : kBlockZ == 1 ? frame_axis(b.a0[d], s.D[d])
                                                : (long long)(b.a0[d] + kBlockZ / 2) * s.D[d];
            const long long fr = frame_axis(aa, s.D[d]) + wrap;
            const long long delta = fr - fb;
            const float hi = i64_to_f32(delta) * s.sx;
            const long long rest = delta - f32_to_i64(hi * pow2f(s.kexp));
            R.hi[tid][d] = hi;
            R.lo[tid][d] = i64_to_f32(rest) * s.sx;
            R.fr[tid][d] = fr;
        }
        const int nb = (a[2] * s.nc[1] + a[1]) * s.nc[0] + a[0];
        const int st = s.cell_start[nb];
        cnt = s.cell_start[nb + 1] - st;
        R.start[tid] = st;
        R.cnt[tid] = cnt;
    }
    // every lane of the warps that cover the region takes part in the scan (lanes past the
    // region carry a count of zero)
    int incl = cnt;
    if (tid < ((kRegion + 31) & ~31)) {
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wtot[tid >> 5] = incl;
    }
    __syncthreads();
    if (tid < kRegion) {
        int base = 0;
        for (int k = 0; k < (tid >> 5); ++k) base += wtot[k];
        int ex = base + incl - cnt;
        R.off[tid] = min(ex, s.smax);
        if (tid == kRegion - 1) {
            int total = base + incl;
            R.off[kRegion] = min(total, s.smax);
            R.nstaged = min(total, s.smax);
            if (total > s.smax) set_status(s, ST_STENCIL_OVERFLOW);
        }
    }
    __syncthreads();
}

// Start staging block b into sm (mixed precision): describe its region, then one TMA bulk
// copy per region cell of the raw frame-relative records, counted on mbar.  Does not wait.
// All threads of the CTA call it; the previous reads of sm must be complete (barrier).
__device__ void issue_block(const DevSim& s, const BlockPos& b, Region& R, float4* sm,
                            uint64_t* mbar) {
    fence_proxy_async_smem();  // earlier generic accesses of sm before the async writes
    region_info(s, b, R);
    const int tid = threadIdx.x;
    if (tid == 0) mbar_arrive_expect_tx(mbar, (uint32_t)R.nstaged * 16u);
    __syncthreads();
    if (tid < kRegion) {
        const int n = R.off[tid + 1] - R.off[tid];
        if (n > 0) bulk_g2s(sm + R.off[tid], s.rel + R.start[tid], (uint32_t)n * 16u, mbar);
    }
}

// Wait for the copies of a block issued with issue_block, add the frame offsets of every
// region cell (exact residual first), write the sentinel sm[smax] and synchronise.
// Returns false on every thread of the CTA if some thread's wait gave up.
__device__ bool finish_block(const DevSim& s, const Region& R, float4* sm, uint64_t* mbar,
                             uint32_t parity) {
    const bool ok = mbar_wait_bounded(s, mbar, parity);
    if (__syncthreads_or(!ok)) return false;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int q = w; q < kRegion; q += kBW) {
        const int o0 = R.off[q], cq = R.off[q + 1] - o0;
        const float hx = R.hi[q][0], hy = R.hi[q][1], hz = R.hi[q][2];
        const float lx = R.lo[q][0], ly = R.lo[q][1], lz = R.lo[q][2];
        for (int t = lane; t < cq; t += 32) {
            float4 v = sm[o0 + t];
            v.x = (v.x + lx) + hx;
            v.y = (v.y + ly) + hy;
            v.z = (v.z + lz) + hz;
            sm[o0 + t] = v;
        }
    }
    if (tid == 0) sm[s.smax] = make_float4(kFar, kFar, kFar, 0.f);
    __syncthreads();
    return true;
}

#ifndef BBMD_STAGE_BUFFERS
#define BBMD_STAGE_BUFFERS 1  // 2: stage block i+1 while block i is computed
#endif
constexpr int kStageBuffers = BBMD_STAGE_BUFFERS;

// Blocks of this CTA in order (grid-stride).  With two staging buffers the copies of block
// i+1 are in flight while block i is computed; with one, each block is staged then
// computed.  body(pos, R, sm) computes one staged block and must not synchronise the CTA.
template <class Body>
__device__ void for_each_block(const DevSim& s, int lb, int lg, float4* smem, int buf_stride, Region* R,
                               uint64_t* mbar, Body body) {
    int64_t blk = lb;
    if (kStageBuffers == 1) {
        for (int it = 0; blk < s.nblocks; ++it, blk += lg) {
            const BlockPos bp = block_pos(s, blk);
            issue_block(s, bp, R[0], smem, &mbar[0]);
            if (!finish_block(s, R[0], smem, &mbar[0], (uint32_t)(it & 1))) return;
            body(bp, R[0], smem);
            __syncthreads();
        }
        return;
    }
    float4* buf[2] = {smem, smem + buf_stride};
    if (blk < s.nblocks) issue_block(s, block_pos(s, blk), R[0], buf[0], &mbar[0]);
    for (int it = 0; blk < s.nblocks; ++it, blk += lg) {
        const int cur = it & 1;
        const int64_t nb = blk + lg;
        if (nb < s.nblocks) issue_block(s, block_pos(s, nb), R[cur ^ 1], buf[cur ^ 1], &mbar[cur ^ 1]);
        if (!finish_block(s, R[cur], buf[cur], &mbar[cur], (uint32_t)((it >> 1) & 1))) {
            // let the copies already issued for the next block land before leaving
            if (nb < s.nblocks)
                mbar_wait_bounded(s, &mbar[cur ^ 1], (uint32_t)(((it + 1) >> 1) & 1));
            return;
        }
        body(block_pos(s, blk), R[cur], buf[cur]);
        __syncthreads();  // buf[cur] and R[cur] are refilled two iterations later
    }
}

// Particles of region cell q that were staged: all of them unless the region overflowed
// the staged capacity (flagged, the results are then discarded), so a lane never reads
// past the staged records.
__device__ __forceinline__ int staged_count(const Region& R, int q) {
    return min(R.cnt[q], R.off[q + 1] - R.off[q]);
}

// Global index of staged entry t (rare path): binary search of the region prefix.
__device__ __forceinline__ int64_t staged_global(const Region& R, int t) {
    int lo = 0, hi = kRegion - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (R.off[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return (int64_t)R.start[lo] + (t - R.off[lo]);
}

// The warp's own cell: its region index and whether it exists (odd nc leaves some warps of
// the last block along an axis idle).
struct WarpCell {
    int c;      // cell id
    int rq;     // region index of the cell
    int wr[3];  // region coordinates of the stencil's first cell per axis
    bool valid;
};

__device__ __forceinline__ WarpCell warp_cell(const DevSim& s, const BlockPos& b, int w) {
    WarpCell wc;
    const int o[3] = {w % kBlockXY, (w / kBlockXY) % kBlockXY, w / (kBlockXY * kBlockXY)};
    int a[3];
    wc.valid = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        a[d] = b.a0[d] + o[d];
        if (a[d] >= s.nc[d]) wc.valid = false;
        wc.wr[d] = o[d];
    }
    wc.c = wc.valid ? (a[2] * s.nc[1] + a[1]) * s.nc[0] + a[0] : 0;
    wc.rq = ((1 + o[2]) * kRXY + (1 + o[1])) * kRXY + (1 + o[0]);
    return wc;
}

// Per-lane pair constants for the lane's species; field suffix = species of j.  Kept as
// scalars and picked with selects so that nothing is indexed at run time.
struct LaneTab {
    float rlo0, rlo1, rhi0, rhi1, sig20, sig21, e480, e481;
    float e40, e41, vsh0, vsh1, fc0, fc1, rc0, rc1, sgl0, sgl1;
    float cpot;   // 0.5 for LJ force, 0 for soft sphere
    float cpe;    // 1 for LJ energy, 0 for soft sphere
    float rm0, rm1, hw;  // list mode: middle of the band around rc^2, half-width (both j)
    int si;
};

__device__ __forceinline__ void load_tab(const DevSim& s, int si, LaneTab& T) {
    const int k = si * 2;
    T.rlo0 = s.pt.rc2lo[k];      T.rlo1 = s.pt.rc2lo[k + 1];
    T.rhi0 = s.pt.rc2hi[k];      T.rhi1 = s.pt.rc2hi[k + 1];
    T.rm0 = 0.5f * (T.rlo0 + T.rhi0);
    T.rm1 = 0.5f * (T.rlo1 + T.rhi1);
    T.hw = 0.5f * fmaxf(T.rhi0 - T.rlo0, T.rhi1 - T.rlo1);
    T.sig20 = s.pt.sig2[k];      T.sig21 = s.pt.sig2[k + 1];
    T.sgl0 = s.pt.sig2lo[k];     T.sgl1 = s.pt.sig2lo[k + 1];
    T.e480 = s.pt.eps48[k];      T.e481 = s.pt.eps48[k + 1];
    T.e40 = s.pt.eps4[k];        T.e41 = s.pt.eps4[k + 1];
    T.vsh0 = s.pt.vshift[k];     T.vsh1 = s.pt.vshift[k + 1];
    T.fc0 = s.pt.fcut[k];        T.fc1 = s.pt.fcut[k + 1];
    T.rc0 = s.pt.frc[k];         T.rc1 = s.pt.frc[k + 1];
    T.cpot = s.pt.potential == BBMD_POT_LJ ? 0.5f : 0.0f;
    T.cpe = s.pt.potential == BBMD_POT_LJ ? 1.0f : 0.0f;
    T.si = si;
}

struct Acc {
    float fx, fy, fz;
};

// Force of one pair; contributes only when `in`.  d = x_j - x_i.  (Pair energies and the
// virial are evaluated by the FP64 energy pass, from exact integer positions.)
template <bool FSHIFT>
__device__ __forceinline__ void pair_add(const LaneTab& T, bool b, float dx, float dy, float dz,
                                         float r2, bool in, Acc& a) {
    float ir2 = rcp_approx(r2);
    float s2 = (b ? T.sig21 : T.sig20) * ir2;
    float s6 = s2 * s2 * s2;
    float f = (b ? T.e481 : T.e480) * ir2 * s6 * (s6 - T.cpot);
    if (FSHIFT) f = fmaf(b ? T.fc1 : T.fc0, rsqrtf(r2), f);
    f = in ? f : 0.f;
    a.fx = fmaf(f, dx, a.fx);
    a.fy = fmaf(f, dy, a.fy);
    a.fz = fmaf(f, dz, a.fz);
}

// Force of one interacting pair with the constants of its species pair given (the stencil
// kernel loads them per candidate stream); the same arithmetic as pair_add.
template <bool FSHIFT>
__device__ __forceinline__ void pair_add_c(float sig2, float e48, float cpot, float fc, float dx, float dy,
                                           float dz, float r2, Acc& a) {
    float ir2 = rcp_approx(r2);
    float s2 = sig2 * ir2;
    float s6 = s2 * s2 * s2;
    float f = e48 * ir2 * s6 * (s6 - cpot);
    if (FSHIFT) f = fmaf(fc, rsqrtf(r2), f);
    a.fx = fmaf(f, dx, a.fx);
    a.fy = fmaf(f, dy, a.fy);
    a.fz = fmaf(f, dz, a.fz);
}

// Fast path of one list pair (i, staged t), classified by d = r^2 - (middle of the band
// around rc^2 for the species of j): interacting iff d <= -hw; |d| < hw is the band,
// left to the exact fix-up; the smallest |d| of a batch tells whether it has band pairs.
template <bool FSHIFT>
__device__ __forceinline__ void pair_fast(const LaneTab& T, float4 me, float4 p, Acc& a, float& near) {
    float dx = p.x - me.x, dy = p.y - me.y, dz = p.z - me.z;
    float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const bool b = p.w != 0.f;
    const float d = r2 - (b ? T.rm1 : T.rm0);
    near = fminf(near, fabsf(d));
    pair_add<FSHIFT>(T, b, dx, dy, dz, r2, d <= -T.hw, a);
}

// A staged copy is usable only in the minimum image (the 4x4x4 region holds a cell twice
// when nc = 3; the two copies are at least a cell side apart from any tile particle).
__device__ __forceinline__ bool min_image_copy(const DevSim& s, float dx, float dy, float dz) {
    return fabsf(dx) < s.halfL[0] && fabsf(dy) < s.halfL[1] && fabsf(dz) < s.halfL[2];
}

// Exact decision for a band pair; adds its force if the FP64 rule says it interacts.  It
// runs for a few pairs per million.  Called out of line (pair_band_call), it keeps the
// lane's pair constants and accumulators in local memory (a stack frame); inline, it
// costs registers.  Inline is faster where the list kernel has 128 registers a thread
// (shapes 4 and 8: 6 % at 2 M particles); out of line where it has fewer (2 x 2 x 1 and
// 2 x 2 x 2: inline is 20 % slower there), and in the persistent batch
// kernel, whose other phases share the register budget (inline, some of its forms spill).
#ifndef BBMD_BAND_INLINE
#define BBMD_BAND_INLINE (BBMD_BLOCK_Z >= 4)
#endif
constexpr bool kBandInline = BBMD_BAND_INLINE;
template <bool FSHIFT>
__device__ __forceinline__ void pair_band(const DevSim& s, const Region& R, const LaneTab& T, float4 me, float4 p,
                          int t, int64_t gi, bool valid, Acc& a) {
    float dx = p.x - me.x, dy = p.y - me.y, dz = p.z - me.z;
    float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const bool b = p.w != 0.f;
    if (!valid || !(fabsf(r2 - (b ? T.rm1 : T.rm0)) < T.hw)) return;
    if (!min_image_copy(s, dx, dy, dz)) return;
    int64_t gj = staged_global(R, t);
    if (r2_exact(s, gi, gj) < s.pt.rc2[T.si * 2 + (b ? 1 : 0)])
        pair_add<FSHIFT>(T, b, dx, dy, dz, r2, true, a);
}

template <bool FSHIFT>
__device__ __noinline__ void pair_band_call(const DevSim& s, const Region& R, const LaneTab& T, float4 me,
                                            float4 p, int t, int64_t gi, bool valid, Acc& a) {
    pair_band<FSHIFT>(s, R, T, me, p, t, gi, valid, a);
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Block reduction of per-warp doubles wv[0 .. nq) (lane 0 of each warp) into
// partials[(q0 + q) * kMaxPartials + lb], in a fixed order.
__device__ void block_partials(const DevSim& s, int lb, const double* wv, int q0, int nq) {
    __shared__ double red[kBW][4];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0)
        for (int q = 0; q < nq; ++q) red[w][q] = wv[q];
    __syncthreads();
    if (threadIdx.x < nq) {
        double t = 0.0;
        for (int k = 0; k < kBW; ++k) t += red[k][threadIdx.x];
        s.partials[(q0 + threadIdx.x) * kMaxPartials + lb] = t;
    }
}

__device__ __forceinline__ unsigned lo16(unsigned w) { return w & 0xffffu; }
__device__ __forceinline__ unsigned hi16(unsigned w) { return w >> 16; }

// Contiguous staged range of stencil row (dy, dz) of the warp's cell: three consecutive
// region cells along x.
__device__ __forceinline__ void stencil_run(const Region& R, const WarpCell& wc, int row, int& rs,
                                            int& re) {
    const int ry = wc.wr[1] + row % 3, rz = wc.wr[2] + row / 3;
    const int q0 = (rz * kRXY + ry) * kRXY + wc.wr[0];
    rs = R.off[q0];
    re = R.off[q0 + 3];
}

// ------------------------------------------------------- stencil compaction ----
// A stencil candidate farther than the reach from the bounding box of the warp's particles
// pairs with none of them.  Such candidates are dropped, 32 at a time, before the per-lane
// tests. The survivors keep their stencil order within their species' stream (below). The
// lists and force sums therefore hold exactly the pairs that testing every candidate finds.
// The reach carries a relative margin of 2^-9. Against it, FP32 rounding of the staged
// coordinates and of the box distance (about 1e-6 relative) is negligible. A dropped
// candidate lies beyond the upper edge of the exact-test band for every lane.

struct WarpBox {
    float lo[3], hi[3];
};

// Shared memory that the force and list bodies use in turn: the staged region's
// description and its mbarriers, and the per-warp candidate rings.  One instance per
// kernel, whichever bodies it runs (a kernel running several bodies, such as the
// persistent batch step, does not pay for each body's own copy).
struct StageShared {
    Region R[kStageBuffers];
    uint64_t mbar[kStageBuffers];
    // the block's work items (cells, or chunks of 32 particles) are handed to the warps in
    // turn as they come free (a count per block parity: one in use, the other reset for
    // the next block)
    int next_cell[2];
    // list-mode chunks of the block: the own particles, species A first then B (each cell
    // holds its A particles first), 32 to a chunk across the block's cells.  Per own cell
    // (in cell order): staged offset, first particle, count, A count; prefixes of the A
    // and B counts; the number of A chunks and of all chunks.
    int c_off[kCells], c_i0[kCells], c_n[kCells], c_nA[kCells];
    int prefA[kCells + 1], prefB[kCells + 1];
    int nchA, nch;
    // kinetic energy of the CTA's chunks in 2^-32 fixed point: integer sums do not depend
    // on which warp added which chunk when
    unsigned long long ke_fix;
};

// Lane `lane` of list-mode chunk `item` of the block: the particle's ordinal o among the
// block's particles of the chunk's species, its cell q (the last whose prefix is <= o: a
// cell with particles), its global index gi and staged index self.
__device__ __forceinline__ void chunk_lane(const StageShared& ss, int item, int lane, bool& act,
                                           int64_t& gi, int& self) {
    const bool isB = item >= ss.nchA;
    const int o = (isB ? item - ss.nchA : item) * 32 + lane;
    const int* pref = isB ? ss.prefB : ss.prefA;
    act = o < pref[kCells];
    int q = 0, hi = kCells - 1;
    while (q < hi) {
        const int mid = (q + hi + 1) >> 1;
        if (pref[mid] <= o) q = mid;
        else hi = mid - 1;
    }
    const int li = (isB ? ss.c_nA[q] : 0) + (o - pref[q]);
    gi = act ? (int64_t)ss.c_i0[q] + li : 0;
    self = act ? ss.c_off[q] + li : 0;
}

// The next work item of the block for this warp (at least the item count when none is
// left).
__device__ __forceinline__ int take_cell(StageShared& ss, int par, int lane) {
    int cw = 0;
    if (lane == 0) cw = atomicAdd(&ss.next_cell[par], 1);
    return __shfl_sync(0xffffffffu, cw, 0);
}

__device__ __forceinline__ StageShared& stage_shared() {
    __shared__ __align__(16) StageShared ss;
    return ss;
}

// Bounding box of the active lanes' positions.
__device__ __forceinline__ WarpBox warp_box(float4 me, bool act) {
    WarpBox b;
    b.lo[0] = act ? me.x : kFar;
    b.lo[1] = act ? me.y : kFar;
    b.lo[2] = act ? me.z : kFar;
    b.hi[0] = act ? me.x : -kFar;
    b.hi[1] = act ? me.y : -kFar;
    b.hi[2] = act ? me.z : -kFar;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            b.lo[d] = fminf(b.lo[d], __shfl_xor_sync(FULL, b.lo[d], o));
            b.hi[d] = fmaxf(b.hi[d], __shfl_xor_sync(FULL, b.hi[d], o));
        }
    }
    return b;
}

// Position in the warp's 27-cell stencil: row (dy, dz) and the next group start g0 in the
// row's staged range [., re).
struct StencilScan {
    int row, g0, re;
};

// Advance to the next non-empty row if the current one is exhausted; false at the end.
__device__ __forceinline__ bool scan_next(const Region& R, const WarpCell& wc, StencilScan& sc) {
    while (sc.g0 >= sc.re) {
        if (++sc.row == 9) return false;
        stencil_run(R, wc, sc.row, sc.g0, sc.re);
    }
    return true;
}

// Squared reach from the box for a candidate of species 0 / 1: the largest upper band edge
// over the lane species, widened by 2^-9.
__device__ __forceinline__ float keep_reach(const float* hi4, int sj) {
    return fmaxf(hi4[sj], hi4[2 + sj]) * (1.0f + 0x1p-9f);
}

// ------------------------------------------------- species-split candidate streams ----
// The list build compacts the stencil candidates within reach of the warp's box into two
// streams, one per species of the candidate.  An entry holds the candidate relative to the
// box centre c, p' = p - c, and q = |p'|^2; a parallel ring holds its staged index.  A
// lane (m' = its own position - c) then tests a candidate of stream S as
//     r^2 - R^2(s_i, S) = q + (|m'|^2 - R^2(s_i, S)) - 2 p'.m'
// (an add and three FMAs after one broadcast load; the threshold is the same for the
// whole stream).  Relative to the box centre, |p'| stays below the box half-diagonal plus
// the reach (about 6 cell sides' worth of r^2 at most), so the FP32 error of this form is
// about 1e-5 in r^2, below the margin of the exact-test band (the band's edges lie at a
// relative 1e-5 and 3e-5 from R^2, about 8e-5 and 2.4e-4 at the bench's R^2 = 7.84).
// The band test uses the same form, so the candidates it sends to the exact rule are
// exactly those whose FP32 value could be on the wrong side.
constexpr int kSRing = 64;  // entries per stream ring (two 32-entry words; a power of two)

struct StreamRings {
    float4 rec[2][kSRing];     // (p' - c, q)
    uint16_t idx[2][kSRing];   // staged index
    float4 box[2];             // (c, reach^2 of species A), (half-extents, reach^2 of B)
};

__device__ __forceinline__ StreamRings& warp_streams(int w) {
    __shared__ __align__(16) StreamRings rings_all[kBW];
    return rings_all[w];
}

// The warp's box as centre and half-extents, kept with the reaches in the warp's
// shared-memory slot (the compaction reads them there: fewer live registers); returns the
// centre.
__device__ __forceinline__ float4 warp_frame(const WarpBox& b, float keepA, float keepB, StreamRings& SR,
                                             int lane) {
    const float4 c = make_float4(0.5f * (b.lo[0] + b.hi[0]), 0.5f * (b.lo[1] + b.hi[1]),
                                 0.5f * (b.lo[2] + b.hi[2]), keepA);
    if (lane == 0) {
        SR.box[0] = c;
        SR.box[1] = make_float4(0.5f * (b.hi[0] - b.lo[0]), 0.5f * (b.hi[1] - b.lo[1]),
                                0.5f * (b.hi[2] - b.lo[2]), keepB);
    }
    __syncwarp();
    return c;
}

// Candidates g0 + lane (below re) go through the box test (against the centred box, with
// the reach of the candidate's species); survivors are appended to their species' stream
// at positions fill[S], fill[S] + 1, ... in candidate order.  cself receives the stream
// position of the lane's own particle (in the stream of its own species) when its group
// passes.
__device__ __forceinline__ void compact_streams(const float4* sm, int g0, int re, StreamRings& SR,
                                                int fill[2], int self, int& cself, int lane) {
    const int t = g0 + lane;
    bool keep = false;
    int sj = 0;
    float4 rec = make_float4(0.f, 0.f, 0.f, 0.f);
    if (t < re) {
        const float4 p = sm[t];
        const float4 c = SR.box[0], h = SR.box[1];
        const float x = p.x - c.x, y = p.y - c.y, z = p.z - c.z;
        const float ex = fmaxf(fabsf(x) - h.x, 0.f);
        const float ey = fmaxf(fabsf(y) - h.y, 0.f);
        const float ez = fmaxf(fabsf(z) - h.z, 0.f);
        sj = p.w != 0.f ? 1 : 0;
        keep = fmaf(ez, ez, fmaf(ey, ey, ex * ex)) < (sj ? h.w : c.w);
        rec = make_float4(x, y, z, fmaf(z, z, fmaf(y, y, x * x)));
    }
    const unsigned bA = __ballot_sync(FULL, keep && sj == 0);
    const unsigned bB = __ballot_sync(FULL, keep && sj == 1);
    const unsigned lt = (1u << lane) - 1u;
    const int pos = sj ? fill[1] + __popc(bB & lt) : fill[0] + __popc(bA & lt);
    if (keep) {
        SR.rec[sj][pos & (kSRing - 1)] = rec;
        SR.idx[sj][pos & (kSRing - 1)] = (uint16_t)t;
    }
    const int src = self - g0;
    const int sp = __shfl_sync(FULL, pos, src & 31);
    if (src >= 0 && src < 32) cself = sp;
    fill[0] += __popc(bA);
    fill[1] += __popc(bB);
}

// After the last group: the rest of stream S's last word holds far records (q huge, so
// every test is positive) pointing at the sentinel.
__device__ __forceinline__ void stream_pad(StreamRings& SR, int S, int fill, int lane, int sentinel) {
    const int pe = (fill + 31) & ~31;
    if (fill + lane < pe) {
        SR.rec[S][(fill + lane) & (kSRing - 1)] = make_float4(kFar, kFar, kFar, 3.0f * kFar * kFar);
        SR.idx[S][(fill + lane) & (kSRing - 1)] = (uint16_t)sentinel;
    }
}

// r^2 - R^2 of a stream entry for a lane: m2 = -2 m', cst = |m'|^2 - R^2(s_i, S).
__device__ __forceinline__ float stream_d(const float4 r, float m2x, float m2y, float m2z, float cst) {
    return fmaf(r.z, m2z, fmaf(r.y, m2y, fmaf(r.x, m2x, r.w + cst)));
}

// Which force kernel runs: in cell mode the stencil kernel (MODE 1); in Verlet mode the
// list kernel (MODE 0), or the stencil kernel while the stored lists are cut at the
// capacity (exact forces until the host has grown the lists).
template <int MODE>
__device__ __forceinline__ bool force_selected(const DevSim& s) {
    if (s.nbr_mode != BBMD_NBR_VERLET) return MODE == 1;
    return (s.sc->list_short != 0) == (MODE == 1);
}

// MODE 0: Verlet list.  MODE 1: every particle of the 27-cell stencil (no stored list).
// BAND_INL: the band fix-up inline (else called out of line).
template <int MODE, bool KE, bool FSHIFT, bool BAND_INL = kBandInline>
__device__ __forceinline__ void force_body(const DevSim& s, int lb, int lg) {
    if (!force_selected<MODE>(s)) return;  // CTA-uniform, before any barrier
    extern __shared__ float4 smem[];
    StageShared& ss = stage_shared();
    Region* const R = ss.R;
    uint64_t* const mbar = ss.mbar;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int k = 0; k < kStageBuffers; ++k) mbar_init(&mbar[k], 1);
        ss.next_cell[0] = ss.next_cell[1] = 0;
        ss.ke_fix = 0ull;
    }
    __syncthreads();
    int blk_it = 0;  // blocks of this CTA so far (the parity selects the counter)
    float hdt0 = 0.f, hdt1 = 0.f;
    if (KE) {
        hdt0 = s.sc->hdt[0];
        hdt1 = s.sc->hdt[1];
    }
    const float m0 = s.pt.mass[0], m1 = s.pt.mass[1];
    const float far = kFar;
    const unsigned sv = (unsigned)s.smax | ((unsigned)s.smax << 16);
    const uint4 sent = make_uint4(sv, sv, sv, sv);
    StreamRings* SRp = nullptr;  // candidate streams of the stencil mode
    if constexpr (MODE == 1) SRp = &warp_streams(w);
    for_each_block(s, lb, lg, smem, s.smax + 1, R, mbar,
                   [&](const BlockPos& bp, const Region& Rc,
                                                      const float4* sm) {
        const int par = blk_it & 1;
        if (threadIdx.x == 0) ss.next_cell[par ^ 1] = 0;  // for the next block
        ++blk_it;
        // the block's work items: in list mode its chunks of one species (a lane's list
        // length depends on its species, and a warp runs to its longest list); in stencil
        // mode its cells (the stencil is the cell's)
        int nitems = kCells;
        if constexpr (MODE == 0) {
            for (int cw = w; cw < kCells; cw += kBW) {
                const WarpCell wc = warp_cell(s, bp, cw);
                const int cnt = wc.valid ? staged_count(Rc, wc.rq) : 0;
                const int off = Rc.off[wc.rq];
                int nA = 0;  // the cell's A particles come first
                for (int t = 0; t < cnt; t += 32) {
                    const unsigned b =
                        __ballot_sync(FULL, t + lane < cnt && sm[off + t + lane].w == 0.f);
                    nA += __popc(b);
                    if (b != FULL) break;
                }
                if (lane == 0) {
                    ss.c_off[cw] = off;
                    ss.c_i0[cw] = wc.valid ? Rc.start[wc.rq] : 0;
                    ss.c_n[cw] = cnt;
                    ss.c_nA[cw] = nA;
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                int na = 0, nb = 0;
                for (int c = 0; c < kCells; ++c) {
                    ss.prefA[c] = na;
                    ss.prefB[c] = nb;
                    na += ss.c_nA[c];
                    nb += ss.c_n[c] - ss.c_nA[c];
                }
                ss.prefA[kCells] = na;
                ss.prefB[kCells] = nb;
                ss.nchA = (na + 31) >> 5;
                ss.nch = ss.nchA + ((nb + 31) >> 5);
            }
            __syncthreads();
            nitems = ss.nch;
        }
        for (int item = take_cell(ss, par, lane); item < nitems; item = take_cell(ss, par, lane)) {
            WarpCell wc;
            int i0 = 0, cnt = 32, self0 = 0;
            if constexpr (MODE == 1) {
                wc = warp_cell(s, bp, item);
                i0 = wc.valid ? Rc.start[wc.rq] : 0;
                cnt = wc.valid ? staged_count(Rc, wc.rq) : 0;
                self0 = Rc.off[wc.rq];
            }
            for (int ch = 0; ch * 32 < cnt; ++ch) {
                bool act;
                int64_t gi;
                int self;
                if constexpr (MODE == 0) {
                    chunk_lane(ss, item, lane, act, gi, self);
                    // the chunk a warp takes kBW items later: its first list rows and
                    // velocities go to L2 now, so that its prologue does not wait on DRAM
                    if (item + kBW < nitems) {
                        bool nact;
                        int64_t ngi;
                        int nself;
                        chunk_lane(ss, item + kBW, lane, nact, ngi, nself);
                        if (nact) {
                            const uint4* lq = reinterpret_cast<const uint4*>(s.list) + ngi;
                            prefetch_l2(lq);
                            prefetch_l2(lq + s.npad);
                            prefetch_l2(s.rows + ngi);
                            if (KE) {
                                prefetch_l2(s.v + ngi);
                                prefetch_l2(s.v + s.npad + ngi);
                                prefetch_l2(s.v + 2 * s.npad + ngi);
                            }
                        }
                    }
                } else {
                    const int li = ch * 32 + lane;
                    act = li < cnt;
                    gi = (int64_t)i0 + li;
                    self = self0 + li;
                }
                // issue the long-latency loads first: the first list rows, the velocity
                const uint4* lp = reinterpret_cast<const uint4*>(s.list) + gi;
                const int myrows = MODE == 0 && act ? (int)s.rows[gi] : 0;  // rows of its list
                uint4 e0 = sent, e1 = sent, e2 = sent;
                if (MODE == 0) {
                    if (myrows > 0) e0 = __ldcs(lp);
                    if (myrows > 1) e1 = __ldcs(lp + s.npad);
                    if (kListAhead > 2 && myrows > 2) e2 = __ldcs(lp + 2 * s.npad);
                }
                // (the stencil loop of MODE 1 needs every register: its velocities are read
                // after it)
                long long v0 = 0, v1 = 0, v2 = 0;
                if (KE && act && MODE == 0) {
                    v0 = s.v[gi];
                    v1 = s.v[s.npad + gi];
                    v2 = s.v[2 * s.npad + gi];
                }
                int nkb = myrows;  // the warp runs to its longest list
                if (MODE == 0)
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) nkb = max(nkb, __shfl_xor_sync(FULL, nkb, o));
                float4 me = act ? sm[self] : make_float4(-far, -far, -far, 0.f);
                const int si = me.w != 0.f ? 1 : 0;
                LaneTab T;
                if constexpr (MODE == 0) load_tab(s, si, T);
                Acc a = {0.f, 0.f, 0.f};
                if (MODE == 0) {
                    for (int kb = 0; kb < nkb; ++kb) {
                        const uint4 e = e0;
                        e0 = e1;
                        if (kListAhead > 2) {
                            e1 = e2;
                            e2 = kb + 3 < myrows ? __ldcs(lp + (int64_t)(kb + 3) * s.npad) : sent;
                        } else {
                            e1 = kb + 2 < myrows ? __ldcs(lp + (int64_t)(kb + 2) * s.npad) : sent;
                        }
                        if (kListPrefetch > 0 && kb + kListPrefetch < myrows)
                            prefetch_l2(lp + (int64_t)(kb + kListPrefetch) * s.npad);
                        float near = far;
                        pair_fast<FSHIFT>(T, me, sm[lo16(e.x)], a, near);
                        pair_fast<FSHIFT>(T, me, sm[hi16(e.x)], a, near);
                        pair_fast<FSHIFT>(T, me, sm[lo16(e.y)], a, near);
                        pair_fast<FSHIFT>(T, me, sm[hi16(e.y)], a, near);
                        pair_fast<FSHIFT>(T, me, sm[lo16(e.z)], a, near);
                        pair_fast<FSHIFT>(T, me, sm[hi16(e.z)], a, near);
                        pair_fast<FSHIFT>(T, me, sm[lo16(e.w)], a, near);
                        pair_fast<FSHIFT>(T, me, sm[hi16(e.w)], a, near);
                        const bool band = near < T.hw;
                        if (__any_sync(FULL, band) && band) {
                            const unsigned ws[4] = {e.x, e.y, e.z, e.w};
                            for (int q = 0; q < 8; ++q) {
                                int t = (q & 1) ? hi16(ws[q >> 1]) : lo16(ws[q >> 1]);
                                if constexpr (BAND_INL)
                                    pair_band<FSHIFT>(s, Rc, T, me, sm[t], t, gi, true, a);
                                else
                                    pair_band_call<FSHIFT>(s, Rc, T, me, sm[t], t, gi, true, a);
                            }
                        }
                    }
                } else {
                    // the stencil on the fly: the candidates within reach of the warp's box
                    // go into the two species streams, each stream word is filtered against
                    // the cutoff into a bitmask (as the list build does against rc + skin),
                    // band candidates are decided by the exact rule, then the forces of the
                    // set bits are added (the species of j is that of the stream)
                    StreamRings& SR = *SRp;
                    const float4 fc = warp_frame(warp_box(me, act), keep_reach(s.pt.rc2hi, 0),
                                                 keep_reach(s.pt.rc2hi, 1), SR, lane);
                    const float mx = act ? me.x - fc.x : 0.f, my = act ? me.y - fc.y : 0.f,
                                mz = act ? me.z - fc.z : 0.f;
                    const float m2x = -2.f * mx, m2y = -2.f * my, m2z = -2.f * mz;
                    const float mm = act ? fmaf(mz, mz, fmaf(my, my, mx * mx)) : far;
                    int fill[2] = {0, 0}, done[2] = {0, 0}, cself = -1;
                    // bitmask of the entries of stream S's word at cq inside the cutoff
                    auto filter_word = [&](int S, int cq) -> unsigned {
                        const float4* const rp = SR.rec[S] + (cq & (kSRing - 1));
                        const float cS = mm - s.pt.rc2lo[si * 2 + S];
                        unsigned inw = 0u;
                        float near = far;
#pragma unroll
                        for (int u = 0; u < 32; ++u) {
                            const float d = stream_d(rp[u], m2x, m2y, m2z, cS);
                            inw = __funnelshift_l(__float_as_uint(d), inw, 1);
                            near = fminf(near, fabsf(d));
                        }
                        const int nv = fill[S] - cq;
                        unsigned valid = nv >= 32 ? 0xffffffffu : ~(0xffffffffu >> nv);
                        if (S == si && cself >= cq && cself < cq + 32)
                            valid &= ~(0x80000000u >> (cself - cq));
                        if (!act) valid = 0u;
                        inw &= valid;
                        const float bS = s.pt.rc2hi[si * 2 + S] - s.pt.rc2lo[si * 2 + S];
                        const bool chk = near < bS && valid != 0u;
                        if (__any_sync(FULL, chk) && chk) {
                            unsigned bw = valid;
                            while (bw) {
                                const int u = __clz(bw);
                                bw &= 0x7fffffffu >> u;
                                if (!(fabsf(stream_d(rp[u], m2x, m2y, m2z, cS)) < bS)) continue;
                                const unsigned bit = 0x80000000u >> u;
                                inw &= ~bit;
                                const float4 r = rp[u];
                                if (!min_image_copy(s, fmaf(m2x, 0.5f, r.x), fmaf(m2y, 0.5f, r.y),
                                                    fmaf(m2z, 0.5f, r.z)))
                                    continue;
                                const int t = (int)SR.idx[S][(cq + u) & (kSRing - 1)];
                                const int64_t gj = staged_global(Rc, t);
                                if (r2_exact(s, gi, gj) < s.pt.rc2[si * 2 + S]) inw |= bit;
                            }
                        }
                        return inw;
                    };
                    // the forces of the set bits of stream S's word at cq
                    auto force_word = [&](int S, int cq) {
                        unsigned inw = filter_word(S, cq);
                        const float4* const rp = SR.rec[S] + (cq & (kSRing - 1));
                        // the constants of the species pair (s_i, S)
                        const int k = si * 2 + S;
                        const float sig2 = s.pt.sig2[k], e48 = s.pt.eps48[k];
                        const float fcut = FSHIFT ? s.pt.fcut[k] : 0.f;
                        const float cpot = s.pt.potential == BBMD_POT_LJ ? 0.5f : 0.0f;
                        while (inw) {
                            const int u = __clz(inw);
                            inw &= 0x7fffffffu >> u;
                            const float4 r = rp[u];
                            // p' - m' (0.5 m2 = -m' exactly)
                            const float dx = fmaf(m2x, 0.5f, r.x), dy = fmaf(m2y, 0.5f, r.y),
                                        dz = fmaf(m2z, 0.5f, r.z);
                            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                            pair_add_c<FSHIFT>(sig2, e48, cpot, fcut, dx, dy, dz, r2, a);
                        }
                    };
                    auto flush_full = [&](int S) {
                        if (fill[S] - done[S] >= 32) {
                            force_word(S, done[S]);
                            done[S] += 32;
                            __syncwarp();
                        }
                    };
                    auto flush_last = [&](int S) {
                        if (fill[S] > done[S]) {
                            stream_pad(SR, S, fill[S], lane, s.smax);
                            __syncwarp();
                            force_word(S, done[S]);
                            done[S] += 32;
                            __syncwarp();
                        }
                    };
                    StencilScan sc = {-1, 0, 0};
                    bool more = scan_next(Rc, wc, sc);
                    while (more) {
                        compact_streams(sm, sc.g0, sc.re, SR, fill, self, cself, lane);
                        sc.g0 += 32;
                        more = scan_next(Rc, wc, sc);
                        __syncwarp();
                        flush_full(0);
                        flush_full(1);
                    }
                    flush_last(0);
                    flush_last(1);
                }
                float fx = -a.fx, fy = -a.fy, fz = -a.fz;
                if (act) {
                    if (!(isfinite(fx) && isfinite(fy) && isfinite(fz))) set_status(s, ST_NONFINITE);
                    s.F[gi] = make_float4(fx, fy, fz, 0.f);
                }
                if (KE) {
                    float k = 0.f;
                    if (act) {
                        if (MODE == 1) {
                            v0 = s.v[gi];
                            v1 = s.v[s.npad + gi];
                            v2 = s.v[2 * s.npad + gi];
                        }
                        const float h = si ? hdt1 : hdt0;
                        const float m = si ? m1 : m0;
                        const float vx = fmaf(h, fx, i64_to_f32_fast(v0) * pow2f(-kVelExp));
                        const float vy = fmaf(h, fy, i64_to_f32_fast(v1) * pow2f(-kVelExp));
                        const float vz = fmaf(h, fz, i64_to_f32_fast(v2) * pow2f(-kVelExp));
                        k = 0.5f * m * fmaf(vx, vx, fmaf(vy, vy, vz * vz));
                    }
                    // the chunk's sum in FP64, added to the CTA's in fixed point
                    const double kc = warp_sum_d((double)k);
                    if (lane == 0) atomicAdd(&ss.ke_fix, __double2ull_rn(kc * 0x1p32));
                }
            }
        }
    });
    if (KE) {
        // every warp has passed the last block's closing barrier
        const double acc_ke = threadIdx.x == 0 ? __ull2double_rn(ss.ke_fix) * 0x1p-32 : 0.0;
        block_partials(s, lb, &acc_ke, 0, 1);
    }
}

// ------------------------------------------------------------------ list build ----

// Each lane tests the compacted candidates of its 27-cell stencil, 32 at a time, with
// broadcast shared-memory reads: the sign of r^2 - R2lo(species of j) is shifted into a
// 32-bit word (candidate u lands in bit 31 - u) and the smallest |r^2 - R2lo| of the word
// is kept.  Only a word whose minimum falls inside the band goes through the exact rule,
// candidate by candidate.  The set bits of each word are then written as list offsets,
// two entries per 32-bit store into [kb][npad][8] uint16, at a row pointer advanced once
// per four pairs.

__device__ __forceinline__ void list_build_body(const DevSim& s, int lb, int lg) {
    if (!s.sc->rebuild) return;
    extern __shared__ float4 smem[];
    StageShared& ss = stage_shared();
    Region* const R = ss.R;
    uint64_t* const mbar = ss.mbar;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int lcap = s.lcap8 * 8;
    const int lcap2 = lcap >> 1;  // pair slots per particle
    StreamRings& SR = warp_streams(w);
    if (threadIdx.x == 0) {
        for (int k = 0; k < kStageBuffers; ++k) mbar_init(&mbar[k], 1);
        ss.next_cell[0] = ss.next_cell[1] = 0;
    }
    __syncthreads();
    int blk_it = 0;  // blocks of this CTA so far (the parity selects the cell counter)
    const float far = kFar;
    const unsigned sentpair = (unsigned)s.smax | ((unsigned)s.smax << 16);
    uint32_t* list32 = reinterpret_cast<uint32_t*>(s.list);
    const int64_t rowstep = (int64_t)s.npad * 4;  // uint32 distance between kb rows
    for_each_block(s, lb, lg, smem, s.smax + 1, R, mbar, [&](const BlockPos& bp, const Region& Rc,
                                                           const float4* sm) {
        const int par = blk_it & 1;
        if (threadIdx.x == 0) ss.next_cell[par ^ 1] = 0;  // for the next block
        ++blk_it;
        for (int cw = take_cell(ss, par, lane); cw < kCells; cw = take_cell(ss, par, lane)) {
            const WarpCell wc = warp_cell(s, bp, cw);
            const int i0 = wc.valid ? Rc.start[wc.rq] : 0;
            const int cnt = wc.valid ? staged_count(Rc, wc.rq) : 0;
            const int self0 = Rc.off[wc.rq];
            for (int ch = 0; ch * 32 < cnt; ++ch) {
                const int li = ch * 32 + lane;
                const bool act = li < cnt;
                const int64_t gi = (int64_t)i0 + li;
                const int self = self0 + li;
                float4 me = act ? sm[self] : make_float4(-far, -far, -far, 0.f);
                const int si = me.w != 0.f ? 1 : 0;
                int len = 0;
                unsigned pend = 0u;
                // pair slot wi (entries 2 wi, 2 wi + 1) of this particle:
                // row0[(wi >> 2) * rowstep + (wi & 3)]
                uint32_t* const row0 = list32 + gi * 4;
                // next pair slot wp and the start of its row
                int wp = 0;
                uint32_t* rowp = row0;
                auto put_pair = [&](unsigned v) {
                    if (wp < lcap2) rowp[wp & 3] = v;
                    ++wp;
                    if ((wp & 3) == 0) rowp += rowstep;
                };
                const float4 fc = warp_frame(warp_box(me, act), keep_reach(s.pt.R2hi, 0),
                                             keep_reach(s.pt.R2hi, 1), SR, lane);
                // the lane relative to the box centre, and its constants per stream
                const float mx = act ? me.x - fc.x : 0.f, my = act ? me.y - fc.y : 0.f,
                            mz = act ? me.z - fc.z : 0.f;
                const float m2x = -2.f * mx, m2y = -2.f * my, m2z = -2.f * mz;
                const float mm = act ? fmaf(mz, mz, fmaf(my, my, mx * mx)) : far;
                int fill[2] = {0, 0}, done[2] = {0, 0}, cself = -1;
                // bitmask of the entries of stream S's word at cq (a multiple of 32) that
                // enter this particle's list (entry u in bit 31 - u)
                auto test_word = [&](int S, int cq) -> unsigned {
                    const float4* const rp = SR.rec[S] + (cq & (kSRing - 1));
                    const float cS = mm - s.pt.R2lo[si * 2 + S];
                    unsigned inw = 0u;
                    float near = far;
#pragma unroll
                    for (int u = 0; u < 32; ++u) {
                        const float d = stream_d(rp[u], m2x, m2y, m2z, cS);
                        inw = __funnelshift_l(__float_as_uint(d), inw, 1);
                        near = fminf(near, fabsf(d));
                    }
                    const int nv = fill[S] - cq;
                    unsigned valid = nv >= 32 ? 0xffffffffu : ~(0xffffffffu >> nv);
                    if (S == si && cself >= cq && cself < cq + 32)
                        valid &= ~(0x80000000u >> (cself - cq));
                    if (!act) valid = 0u;
                    inw &= valid;
                    const float bS = s.pt.R2hi[si * 2 + S] - s.pt.R2lo[si * 2 + S];
                    const bool chk = near < bS && valid != 0u;
                    if (__any_sync(FULL, chk) && chk) {
                        // the same FP32 value decides which entries are in the band; those
                        // are decided by the exact rule
                        unsigned bw = valid;
                        while (bw) {
                            const int u = __clz(bw);
                            bw &= 0x7fffffffu >> u;
                            if (!(fabsf(stream_d(rp[u], m2x, m2y, m2z, cS)) < bS)) continue;
                            const unsigned bit = 0x80000000u >> u;
                            inw &= ~bit;
                            // (p' - m' is the separation up to FP32 rounding: enough to tell
                            // the minimum-image copy from one a box length away)
                            const float4 r = rp[u];
                            if (!min_image_copy(s, fmaf(m2x, 0.5f, r.x), fmaf(m2y, 0.5f, r.y),
                                                fmaf(m2z, 0.5f, r.z)))
                                continue;
                            const int t = (int)SR.idx[S][(cq + u) & (kSRing - 1)];
                            const int64_t gj = staged_global(Rc, t);
                            if (r2_exact(s, gi, gj) < s.pt.R2[si * 2 + S]) inw |= bit;
                        }
                    }
                    return inw;
                };
                // the set bits of stream S's word at cq as list entries, in stream order
                auto append_word = [&](int S, int cq, unsigned bits) {
                    // the word's 32 entries are contiguous (word starts are multiples of 32
                    // in a ring of 64)
                    const uint16_t* const rw = SR.idx[S] + (cq & (kSRing - 1));
                    // entries go out in pairs (one 32-bit store each at the running row
                    // pointer; entries beyond the capacity are counted, not stored): a
                    // pending odd entry is completed by the word's first bit, then two
                    // bits per iteration; an odd last bit stays pending
                    if ((len & 1) && bits) {
                        const int u = __clz(bits);
                        bits &= 0x7fffffffu >> u;
                        put_pair(pend | ((unsigned)rw[u] << 16));
                        ++len;
                    }
                    while (bits) {
                        const int u1 = __clz(bits);
                        bits &= 0x7fffffffu >> u1;
                        const unsigned t1 = rw[u1];
                        if (!bits) {
                            pend = t1;
                            ++len;
                            break;
                        }
                        const int u2 = __clz(bits);
                        bits &= 0x7fffffffu >> u2;
                        put_pair(t1 | ((unsigned)rw[u2] << 16));
                        len += 2;
                    }
                };
                // a stream's word is tested and appended as soon as it is full (fewer than
                // 32 entries wait in each ring before a group adds at most 32)
                auto flush_full = [&](int S) {
                    if (fill[S] - done[S] >= 32) {
                        append_word(S, done[S], test_word(S, done[S]));
                        done[S] += 32;
                        __syncwarp();
                    }
                };
                StencilScan sc = {-1, 0, 0};
                bool more = scan_next(Rc, wc, sc);
                while (more) {
                    compact_streams(sm, sc.g0, sc.re, SR, fill, self, cself, lane);
                    sc.g0 += 32;
                    more = scan_next(Rc, wc, sc);
                    __syncwarp();
                    flush_full(0);
                    flush_full(1);
                }
                // the partial last word of each stream
                auto flush_last = [&](int S) {
                    if (fill[S] > done[S]) {
                        stream_pad(SR, S, fill[S], lane, s.smax);
                        __syncwarp();
                        append_word(S, done[S], test_word(S, done[S]));
                        done[S] += 32;
                        __syncwarp();
                    }
                };
                flush_last(0);
                flush_last(1);
                if (len > lcap) {
                    // the list is cut: flagged for the host (which grows the capacity at its
                    // next synchronising call) and, until then, the forces come from the
                    // cell stencil
                    set_status(s, ST_LIST_OVERFLOW);
                    s.sc->list_short = 1;
                    atomicMax(&s.sc->max_len, len);
                    len = lcap;
                }
                if (act && (len & 1)) {
                    const int wi = len >> 1;
                    row0[(int64_t)(wi >> 2) * rowstep + (wi & 3)] = pend | ((unsigned)s.smax << 16);
                    ++len;
                }
                if (act) {
                    // the rest of the last row holds sentinel pairs; the particle's row count
                    // tells the force kernels where its list ends
                    const int rows = (len + 7) >> 3;
                    for (int wi = len >> 1; wi < rows * 4; ++wi)
                        row0[(int64_t)(wi >> 2) * rowstep + (wi & 3)] = sentpair;
                    s.rows[gi] = (uint16_t)rows;
                }
            }
        }
    });
}

// ------------------------------------------------------- persistent batch step ----
// One cooperative launch advances every replica of a batch by many steps.  The step of
// each replica is a chain of phases (integrate, the two trigger passes, the seven sort
// passes, the list build, forces, finalize); each phase of each replica is cut into work
// items with the same (CTA index, CTA count) as the kernels launched for one system, so a
// replica advances bit for bit as it would alone.  The items of all replicas are handed
// out from one queue, step after step and phase-major within a step: a CTA takes the next
// item, waits until the replica's previous non-empty phase is complete (for the first
// phase of a step: the finalize of the replica's previous step) by a per-replica,
// per-phase count of finished items (bounded), runs the item and counts it finished.
// Replicas never wait on each other, so the phases and steps of different replicas
// overlap; an item waits only on items handed out before it, and every CTA is resident,
// so the queue always advances.
#if BBMD_BLOCK_Z == BBMD_PERSIST_Z
#include "sort_bodies.cuh"
#include "step_bodies.cuh"

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Raise the abort flag and ST_TIMEOUT on every replica.
__device__ __forceinline__ void persistent_abort(const PersistentStep& a) {
    if (atomicExch(a.abort, 1) == 0)
        for (int r = 0; r < a.nrep; ++r) atomicOr(&a.sims[r].sc->status, ST_TIMEOUT);
}

template <bool KE, bool FSHIFT>
__device__ __forceinline__ void run_phase(int phase, const DevSim& s, int lb, int lg) {
    switch (phase) {
        case kPhIntegrate: integrate_body<false>(s, lb, lg); break;
        case kPhCelltop: celltop_body(s, lb, lg); break;
        case kPhCheck: check_body(s, lb, lg); break;
        case kPhZero: zero_body(s, lb, lg); break;
        case kPhBin: bin_body(s, lb, lg); break;
        case kPhScan: scan_cta_body(s, lb, lg); break;
        case kPhScatter: scatter_body(s, lb, lg); break;
        case kPhCellsort: cellsort_body(s, lb, lg); break;
        case kPhGather: gather_body(s, lb, lg); break;
        case kPhCopyback: copyback_body(s, lb, lg); break;
        case kPhList: list_build_body(s, lb, lg); break;
        case kPhForce:
            // the list body, or for a replica whose lists are cut (and in cell mode) the
            // stencil body: each returns at once when not selected
            force_body<0, KE, FSHIFT, false>(s, lb, lg);
            force_body<1, KE, FSHIFT, false>(s, lb, lg);
            break;
        default: finalize_body(s, KE ? 1 : 0); break;
    }
}

template <bool KE, bool FSHIFT>
__global__ void __launch_bounds__(kBW * 32, 2) k_step_persistent(PersistentStep a) {
    __shared__ DevSim sh;
    __shared__ int4 desc;  // phase, replica, lb, lg of the item (phase -1: queue empty)
    __shared__ int run;    // 0: the item's replica does not rebuild (gated phase)
    for (;;) {
        if (threadIdx.x == 0) {
            int4 d = make_int4(-1, 0, 0, 0);
            int go = 0;
            if (*(volatile int*)a.abort == 0) {
                const long long k = (long long)atomicAdd(a.head, 1u);
                if (k < (long long)a.nitems * a.nsteps) {
                    const int step = (int)(k / a.nitems);
                    d = a.items[k - (long long)step * a.nitems];
                    int dep = a.dep[d.y * kPhases + d.x], dstep = step;
                    if (dep < 0 && step > 0) {
                        dep = kPhFinalize;  // the replica's previous step
                        dstep = step - 1;
                    }
                    if (dep >= 0) {
                        const int need = a.need[d.y * kPhases + dep] * (dstep + 1);
                        const int* cnt = &a.done[d.y * kPhases + dep];
                        const unsigned long long t0 = globaltimer_ns();
                        while (*(volatile const int*)cnt < need) {
                            if (*(volatile int*)a.abort) {
                                d.x = -1;
                                break;
                            }
                            if (globaltimer_ns() - t0 > a.wait_ns) {
                                persistent_abort(a);
                                d.x = -1;
                                break;
                            }
                        }
                        __threadfence();
                    }
                    go = d.x >= 0;
                    if (go && d.x >= kPhZero && d.x <= kPhList)
                        go = *(volatile int*)&a.sims[d.y].sc->rebuild != 0;
                }
            }
            desc = d;
            run = go;
        }
        __syncthreads();
        const int4 d = desc;
        if (d.x < 0) return;
        // data of earlier phases, written by other CTAs, is read by bulk copies (the async
        // proxy) as well as by ordinary loads
        asm volatile("fence.proxy.async.global;" ::: "memory");
        if (run) {
            const int4* src4 = reinterpret_cast<const int4*>(a.sims + d.y);
            int4* dst4 = reinterpret_cast<int4*>(&sh);
            for (int k = threadIdx.x; k < (int)(sizeof(DevSim) / 16); k += blockDim.x) dst4[k] = src4[k];
            __syncthreads();
            run_phase<KE, FSHIFT>(d.x, sh, d.z, d.w);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&a.done[d.y * kPhases + d.x], 1);
        }
    }
}
#endif  // BBMD_BLOCK_Z == BBMD_PERSIST_Z

// ------------------------------------------------------------------ FP64 form ----
// The same block region staged as exact integer positions in the block's periodic image
// (frame point + seam image + the particle's minimum-image offset from the frame, which
// stays right after the particle itself has crossed the boundary since the last build);
// distances are the exact integer differences rounded once to double (the rule the list
// decisions use), pair arithmetic and accumulation in FP64.

struct Pos64 {
    long long x, y, z;
    int sp, pad;
};

__device__ void stage_block64(const DevSim& s, const BlockPos& b, Region& R, Pos64* sm) {
    region_info(s, b, R);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int q = w; q < kRegion; q += kBW) {
        const int o0 = R.off[q], cq = R.off[q + 1] - o0;
        const long long fx = R.fr[q][0], fy = R.fr[q][1], fz = R.fr[q][2];
        for (int t = lane; t < cq; t += 32) {
            const int64_t j = R.start[q] + t;
            Pos64 p;
            p.x = fx + min_image((long long)s.x[j] - fx, s.Lfix[0]);
            p.y = fy + min_image((long long)s.x[s.npad + j] - fy, s.Lfix[1]);
            p.z = fz + min_image((long long)s.x[2 * s.npad + j] - fz, s.Lfix[2]);
            p.sp = s.sp[j];
            p.pad = 0;
            sm[o0 + t] = p;
        }
    }
    if (threadIdx.x == 0) {
        // staged positions lie in (-L_fix, 2 L_fix) with L_fix < 2^62: a sentinel at 3 * 2^61
        // on every axis is beyond every cutoff (|dx| > L/2 is never a minimum image) and no
        // difference overflows
        Pos64 far;
        far.x = far.y = far.z = (long long)3 << 61;
        far.sp = 0;
        far.pad = 0;
        sm[s.smax] = far;
    }
    __syncthreads();
}

template <bool ENERGY, bool FSHIFT>
__device__ __forceinline__ void pair_fp64(const DevSim& s, int si, const Pos64& me, const Pos64& p,
                                          double& fx, double& fy, double& fz, double& u,
                                          double& w) {
    const long long ix = p.x - me.x, iy = p.y - me.y, iz = p.z - me.z;
    const int k = si * 2 + p.sp;
    // integer pre-test: a separation beyond rc on some axis cannot interact.  rc < L/2 (the
    // box holds at least three cells of side >= rc per axis), so what passes is the
    // minimum-image copy (a region may hold a cell twice when nc = 3)
    const long long lim = s.pt.rcfix[k];
    if (llabs(ix) > lim || llabs(iy) > lim || llabs(iz) > lim) return;
    double dx = __dmul_rn(__ll2double_rn(ix), s.sxd);
    double dy = __dmul_rn(__ll2double_rn(iy), s.sxd);
    double dz = __dmul_rn(__ll2double_rn(iz), s.sxd);
    double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    if (r2 < s.pt.rc2[k]) {
        double ir2 = 1.0 / r2;
        double s2 = s.pt.dsig2[k] * ir2;
        double s6 = s2 * s2 * s2;
        double cp = s.pt.potential == BBMD_POT_LJ ? 0.5 : 0.0;
        double f = s.pt.deps48[k] * ir2 * s6 * (s6 - cp);
        double r = 0.0;
        if (FSHIFT) {
            r = sqrt(r2);
            f += s.pt.dfcut[k] / r;
        }
        fx += f * dx;
        fy += f * dy;
        fz += f * dz;
        if (ENERGY) {
            double ce = s.pt.potential == BBMD_POT_LJ ? 1.0 : 0.0;
            double V = s.pt.deps4[k] * s6 * (s6 - ce) - s.pt.dvshift[k];
            if (FSHIFT) V -= (r - s.pt.drc[k]) * s.pt.dfcut[k];
            u += V;
            w += f * r2;
        }
    }
}

// ENERGY: per-particle energies u_i (half of each pair energy), and the energy and virial
// partials 1 and 2.  EONLY (with ENERGY, mixed precision): the energy pass of a
// mixed-precision handle -- the same exact integer positions and FP64 pair arithmetic,
// but the forces stay those of the FP32 kernel (nothing is written to F or Fd).
template <int MODE, bool ENERGY, bool KE, bool FSHIFT, bool EONLY = false>
__device__ __forceinline__ void force64_body(const DevSim& s, int lb, int lg) {
    if (!force_selected<MODE>(s)) return;  // CTA-uniform, before any barrier
    extern __shared__ float4 smem[];
    __shared__ Region R;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    Pos64* sm = reinterpret_cast<Pos64*>(smem);
    double acc_ke = 0.0, acc_u = 0.0, acc_w = 0.0;
    for (int64_t blk = lb; blk < s.nblocks; blk += lg) {
        const BlockPos bp = block_pos(s, blk);
        stage_block64(s, bp, R, sm);
        for (int cw = w; cw < kCells; cw += kBW) {
        const WarpCell wc = warp_cell(s, bp, cw);
        const int i0 = wc.valid ? s.cell_start[wc.c] : 0;
        const int cnt = wc.valid ? staged_count(R, wc.rq) : 0;
        const int self0 = R.off[wc.rq];
        for (int ch = 0; ch * 32 < cnt; ++ch) {
            const int li = ch * 32 + lane;
            const bool act = li < cnt;
            const int64_t gi = (int64_t)i0 + li;
            Pos64 me;
            if (act) {
                me = sm[self0 + li];
            } else {
                me.x = me.y = me.z = -((long long)1 << 62);
                me.sp = 0;
            }
            const int si = me.sp;
            double fx = 0, fy = 0, fz = 0, u = 0, wv = 0;
            if (MODE == 0) {
                const int nkb = act ? (int)s.rows[gi] : 0;  // rows of the particle's list
                const uint4* lp = reinterpret_cast<const uint4*>(s.list) + gi;
                for (int kb = 0; kb < nkb; ++kb) {
                    uint4 e = lp[(int64_t)kb * s.npad];
                    unsigned ws[4] = {e.x, e.y, e.z, e.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        pair_fp64<ENERGY, FSHIFT>(s, si, me, sm[ws[q] & 0xffffu], fx, fy, fz, u, wv);
                        pair_fp64<ENERGY, FSHIFT>(s, si, me, sm[ws[q] >> 16], fx, fy, fz, u, wv);
                    }
                }
            } else if (act) {
                const int self = self0 + li;
                for (int row = 0; row < 9; ++row) {
                    int rs, re;
                    stencil_run(R, wc, row, rs, re);
                    for (int t = rs; t < re; ++t) {
                        if (t == self) continue;
                        pair_fp64<ENERGY, FSHIFT>(s, si, me, sm[t], fx, fy, fz, u, wv);
                    }
                }
            }
            if (act && !EONLY) {
                fx = -fx;
                fy = -fy;
                fz = -fz;
                if (!(isfinite(fx) && isfinite(fy) && isfinite(fz))) set_status(s, ST_NONFINITE);
                s.Fd[gi] = fx;
                s.Fd[s.npad + gi] = fy;
                s.Fd[2 * s.npad + gi] = fz;
                s.F[gi] = make_float4((float)fx, (float)fy, (float)fz, 0.f);
            }
            if (act && ENERGY) s.ud[gi] = 0.5 * u;
            if (KE) {
                double k = 0.0;
                if (act) {
                    double h = 0.5 * s.sc->dt / s.pt.dmass[si];
                    double vx = __ll2double_rn(s.v[gi]) * 0x1p-52 + h * fx;
                    double vy = __ll2double_rn(s.v[s.npad + gi]) * 0x1p-52 + h * fy;
                    double vz = __ll2double_rn(s.v[2 * s.npad + gi]) * 0x1p-52 + h * fz;
                    k = 0.5 * s.pt.dmass[si] * (vx * vx + vy * vy + vz * vz);
                }
                k = warp_sum_d(k);
                if (lane == 0) acc_ke += k;
            }
            if (ENERGY) {
                double uu = warp_sum_d(act ? 0.5 * u : 0.0);
                double ww = warp_sum_d(act ? 0.5 * wv : 0.0);
                if (lane == 0) {
                    acc_u += uu;
                    acc_w += ww;
                }
            }
        }
        }
        __syncthreads();
    }
    if (EONLY) {
        const double wv2[2] = {acc_u, acc_w};
        block_partials(s, lb, wv2, 1, 2);
    } else if (KE || ENERGY) {
        const double wv3[3] = {acc_ke, acc_u, acc_w};
        block_partials(s, lb, wv3, 0, 3);
    }
}

// ------------------------------------------------------------------ kernels ----
// Each body runs for one system (DevSim by value) or, in the _many form, for the replica of
// a batch that owns the CTA.

template <int MODE, bool KE, bool FSHIFT>
__global__ void __launch_bounds__(kBW * 32, MODE == 1 ? BBMD_CELL_MIN_BLOCKS : BBMD_FORCE_MIN_BLOCKS)
    k_force(DevSim s) {
    force_body<MODE, KE, FSHIFT>(s, (int)blockIdx.x, (int)gridDim.x);
}

template <int MODE, bool KE, bool FSHIFT>
__global__ void __launch_bounds__(kBW * 32, MODE == 1 ? BBMD_CELL_MIN_BLOCKS : BBMD_FORCE_MIN_BLOCKS)
    k_force_many(ManySims m) {
    __shared__ DevSim sh;
    int lb, lg;
    load_replica(m, sh, lb, lg);
    force_body<MODE, KE, FSHIFT>(sh, lb, lg);
}

__global__ void __launch_bounds__(kBW * 32, BBMD_LIST_MIN_BLOCKS) k_list_build(DevSim s) {
    list_build_body(s, (int)blockIdx.x, (int)gridDim.x);
}

__global__ void __launch_bounds__(kBW * 32, BBMD_LIST_MIN_BLOCKS) k_list_build_many(ManySims m) {
    __shared__ DevSim sh;
    int lb, lg;
    load_replica(m, sh, lb, lg);
    list_build_body(sh, lb, lg);
}

template <int MODE, bool ENERGY, bool KE, bool FSHIFT, bool EONLY = false>
__global__ void __launch_bounds__(kBW * 32) k_force64(DevSim s) {
    force64_body<MODE, ENERGY, KE, FSHIFT, EONLY>(s, (int)blockIdx.x, (int)gridDim.x);
}

template <int MODE, bool ENERGY, bool KE, bool FSHIFT>
__global__ void __launch_bounds__(kBW * 32) k_force64_many(ManySims m) {
    __shared__ DevSim sh;
    int lb, lg;
    load_replica(m, sh, lb, lg);
    force64_body<MODE, ENERGY, KE, FSHIFT>(sh, lb, lg);
}

// Opt every kernel with dynamic shared memory into the largest size the device allows
// next to the kernel's static shared memory (done at create, outside any stream capture);
// each launch then requests only what it needs.
static bool g_smem_ok = true;

template <typename K>
void set_smem(K kernel) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) {
        g_smem_ok = false;
        return;
    }
    int dyn = optin - (int)fa.sharedSizeBytes;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) !=
        cudaSuccess)
        g_smem_ok = false;
}

// Mixed precision: FP32 forces; an energy pass (E) adds the FP64 energy kernel, which
// writes the per-particle energies and the energy and virial partials from exact integer
// positions (FP32 coordinates would limit u_i to about 1e-4).
template <int MODE, bool E, bool KE, bool FS>
void run_force(const DevSim& s, cudaStream_t st) {
    const size_t bytes64 = (size_t)(s.smax + 1) * sizeof(Pos64);
    if (s.precision == BBMD_PREC_FP64) {
        k_force64<MODE, E, KE, FS><<<s.grid_cell, kBW * 32, bytes64, st>>>(s);
    } else {
        size_t bytes = kStageBuffers * (size_t)(s.smax + 1) * sizeof(float4);
        k_force<MODE, KE, FS><<<s.grid_cell, kBW * 32, bytes, st>>>(s);
        if (E) k_force64<MODE, true, false, FS, true><<<s.grid_cell, kBW * 32, bytes64, st>>>(s);
    }
}

template <int MODE, bool KE, bool FS>
void run_force_many(const ManySims& m, int total, bool fp64, int smax_max, cudaStream_t st) {
    if (fp64) {
        size_t bytes = (size_t)(smax_max + 1) * sizeof(Pos64);
        k_force64_many<MODE, false, KE, FS><<<total, kBW * 32, bytes, st>>>(m);
    } else {
        size_t bytes = kStageBuffers * (size_t)(smax_max + 1) * sizeof(float4);
        k_force_many<MODE, KE, FS><<<total, kBW * 32, bytes, st>>>(m);
    }
}

template <int MODE>
void run_force_mode(const DevSim& s, cudaStream_t st, bool energy, bool ke, bool fs) {
    if (fs) {
        if (energy) {
            if (ke) run_force<MODE, true, true, true>(s, st); else run_force<MODE, true, false, true>(s, st);
        } else {
            if (ke) run_force<MODE, false, true, true>(s, st); else run_force<MODE, false, false, true>(s, st);
        }
    } else {
        if (energy) {
            if (ke) run_force<MODE, true, true, false>(s, st); else run_force<MODE, true, false, false>(s, st);
        } else {
            if (ke) run_force<MODE, false, true, false>(s, st); else run_force<MODE, false, false, false>(s, st);
        }
    }
}

template <int MODE, bool E, bool KE, bool FS>
void prep_one() {
    set_smem(k_force64<MODE, E, KE, FS>);
    if (E) {
        if (!KE) set_smem(k_force64<MODE, true, false, FS, true>);
    } else {
        set_smem(k_force<MODE, KE, FS>);
        set_smem(k_force_many<MODE, KE, FS>);
        set_smem(k_force64_many<MODE, E, KE, FS>);
    }
}

template <int MODE>
void prep_mode() {
    prep_one<MODE, false, false, false>();
    prep_one<MODE, false, true, false>();
    prep_one<MODE, true, false, false>();
    prep_one<MODE, true, true, false>();
    prep_one<MODE, false, false, true>();
    prep_one<MODE, false, true, true>();
    prep_one<MODE, true, false, true>();
    prep_one<MODE, true, true, true>();
}

}  // namespace

int block_threads() { return kBW * 32; }

bool prepare_force_kernels() {
    g_smem_ok = true;
    prep_mode<0>();
    prep_mode<1>();
    set_smem(k_list_build);
    set_smem(k_list_build_many);
    return g_smem_ok;
}

int force_blocks_per_sm(const DevSim& s) {
    int nb = 0;
    size_t bytes = s.precision == BBMD_PREC_FP64 ? (size_t)(s.smax + 1) * sizeof(Pos64)
                                                 : kStageBuffers * (size_t)(s.smax + 1) * sizeof(float4);
    if (s.precision == BBMD_PREC_FP64)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_force64<0, false, true, false>, kBW * 32, bytes);
    else if (s.nbr_mode == BBMD_NBR_CELL)  // the stencil kernel is the step's force kernel
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_force<1, true, false>, kBW * 32, bytes);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_force<0, true, false>, kBW * 32, bytes);
    return nb > 0 ? nb : 1;
}

int list_blocks_per_sm(const DevSim& s) {
    int nb = 0;
    const size_t bytes = kStageBuffers * (size_t)(s.smax + 1) * sizeof(float4);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_list_build, kBW * 32, bytes);
    return nb > 0 ? nb : 1;
}

// Verlet mode launches the list kernel and, behind it, the stencil kernel: exactly one of
// the two runs, by the device flag of cut lists.
void launch_force(const DevSim& s, cudaStream_t st, bool energy, bool ke) {
    bool fs = s.pt.shift == BBMD_SHIFT_FORCE;
    if (s.nbr_mode == BBMD_NBR_VERLET) run_force_mode<0>(s, st, energy, ke, fs);
    run_force_mode<1>(s, st, energy, ke, fs);
}

void launch_force_many(const ManySims& m, int total, bool fp64, bool cell, bool ke, bool fshift,
                       int smax_max, cudaStream_t st) {
    if (cell) {
        if (ke) {
            if (fshift) run_force_many<1, true, true>(m, total, fp64, smax_max, st);
            else run_force_many<1, true, false>(m, total, fp64, smax_max, st);
        } else {
            if (fshift) run_force_many<1, false, true>(m, total, fp64, smax_max, st);
            else run_force_many<1, false, false>(m, total, fp64, smax_max, st);
        }
    } else {
        // list kernel, then the stencil kernel that stands in for replicas with cut lists
        if (ke) {
            if (fshift) {
                run_force_many<0, true, true>(m, total, fp64, smax_max, st);
                run_force_many<1, true, true>(m, total, fp64, smax_max, st);
            } else {
                run_force_many<0, true, false>(m, total, fp64, smax_max, st);
                run_force_many<1, true, false>(m, total, fp64, smax_max, st);
            }
        } else {
            if (fshift) {
                run_force_many<0, false, true>(m, total, fp64, smax_max, st);
                run_force_many<1, false, true>(m, total, fp64, smax_max, st);
            } else {
                run_force_many<0, false, false>(m, total, fp64, smax_max, st);
                run_force_many<1, false, false>(m, total, fp64, smax_max, st);
            }
        }
    }
}

void launch_list_build_many(const ManySims& m, int total, int smax_max, cudaStream_t st) {
    const size_t bytes = kStageBuffers * (size_t)(smax_max + 1) * sizeof(float4);
    k_list_build_many<<<total, kBW * 32, bytes, st>>>(m);
}

void launch_list_build(const DevSim& s, cudaStream_t st) {
    if (s.nbr_mode != BBMD_NBR_VERLET) return;
    // staging buffer(s), each: staged region + sentinel record
    size_t bytes = kStageBuffers * (size_t)(s.smax + 1) * sizeof(float4);
    k_list_build<<<s.grid_list, kBW * 32, bytes, st>>>(s);
}

#if BBMD_BLOCK_Z == BBMD_PERSIST_Z
// Dynamic shared memory of the persistent step for staged capacity smax_max.
static size_t persistent_smem(int smax_max) {
    return kStageBuffers * (size_t)(smax_max + 1) * sizeof(float4);
}

bool prepare_persistent() {
    g_smem_ok = true;
    set_smem(k_step_persistent<false, false>);
    set_smem(k_step_persistent<true, false>);
    set_smem(k_step_persistent<false, true>);
    set_smem(k_step_persistent<true, true>);
    return g_smem_ok;
}

int persistent_blocks_per_sm(int smax_max) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_persistent<true, false>, kBW * 32,
                                                  persistent_smem(smax_max));
    return nb;
}

cudaError_t launch_persistent_step(const PersistentStep& a, int grid, int smax_max, bool ke,
                                   bool fshift, cudaStream_t st) {
    PersistentStep args = a;
    void* params[] = {&args};
    const void* fn = ke ? (fshift ? (const void*)k_step_persistent<true, true>
                                  : (const void*)k_step_persistent<true, false>)
                        : (fshift ? (const void*)k_step_persistent<false, true>
                                  : (const void*)k_step_persistent<false, false>);
    return cudaLaunchCooperativeKernel(fn, grid, kBW * 32, params, persistent_smem(smax_max), st);
}
#endif  // BBMD_BLOCK_Z == BBMD_PERSIST_Z

}  // namespace z<BBMD_BLOCK_Z>
}  // namespace bbmd
