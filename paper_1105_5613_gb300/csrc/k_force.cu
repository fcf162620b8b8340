// Pair forces of the truncated Lennard-Jones / soft-sphere mixture (Sec. 2.1, Eqs. lj0,
// sc0, mod0) over the cell stencil (Sec. 2.2), and the Verlet-list build.
//
// Work unit: one warp per cell ("tile" = up to 32 particles of the cell; larger cells are
// processed in chunks of 32).  The warp stages the particles of the 27 surrounding cells
// into its shared-memory stencil as float4 {x, y, z, species}, with coordinates expressed
// in the frame of the tile's cell (the frame offset between two cells is exact in FP32
// away from the periodic seam).  Each lane owns one particle i and accumulates its force
// in registers: a full list, one writer per i, no atomics (the paper applies Newton's
// third law to halve the pair work on a CPU; here every pair is visited from both sides
// so that each force has a single owner and a fixed summation order).
//
// The Verlet list stores, per particle, uint16 offsets into the staged stencil; entries
// are laid out as [kb][npad][8] so a warp reads 8 entries per lane with one coalesced
// 16-byte load.  Padding entries point to a sentinel far outside every cutoff.
//
// Mixed precision: distances and forces in FP32 from frame-relative coordinates; a pair
// whose FP32 r^2 lies within a relative 1e-5 of the cutoff is re-tested with the exact
// FP64 rule so that the interacting set equals the FP64 definition.
#include "bbmd_internal.cuh"

namespace bbmd {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr float kFar = 1.0e15f;

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

struct StencilInfo {
    int off[28];   // prefix of staged counts (off[27] = total)
    int cell[27];  // neighbour cell ids (fixed order: dz, dy, dx in -1..1)
};

// Stage the 27-cell stencil of cell c into sm[0 .. total) (+ sentinel at sm[smax]).
// Returns the staged count (truncated to smax, with a status bit on overflow).
__device__ int stage_stencil(const DevSim& s, int c, float4* sm, StencilInfo& st, int lane) {
    int ax, ay, az;
    cell_coords(c, s.nc, ax, ay, az);
    int start = 0, cnt = 0, nb = 0;
    float shx = 0.f, shy = 0.f, shz = 0.f;
    if (lane < 27) {
        int o[3] = {lane % 3 - 1, (lane / 3) % 3 - 1, lane / 9 - 1};
        int a[3] = {ax, ay, az};
        int b[3];
        float sh[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            int bb = a[d] + o[d];
            long long wrap = 0;
            if (bb < 0) {
                bb += s.nc[d];
                wrap = -s.Lfix[d];
            } else if (bb >= s.nc[d]) {
                bb -= s.nc[d];
                wrap = s.Lfix[d];
            }
            b[d] = bb;
            long long delta = frame_axis(bb, s.D[d]) + wrap - frame_axis(a[d], s.D[d]);
            sh[d] = i64_to_f32(delta) * s.sx;
        }
        nb = (b[2] * s.nc[1] + b[1]) * s.nc[0] + b[0];
        start = s.cell_start[nb];
        cnt = s.cell_start[nb + 1] - start;
        shx = sh[0];
        shy = sh[1];
        shz = sh[2];
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += t;
    }
    int total = __shfl_sync(FULL, incl, 26);
    if (lane < 27) {
        st.off[lane] = incl - cnt;
        st.cell[lane] = nb;
    }
    if (lane == 0) st.off[27] = total;
    __syncwarp();
    if (total > s.smax) {
        if (lane == 0) set_status(s, ST_STENCIL_OVERFLOW);
        total = s.smax;
    }
    for (int q = 0; q < 27; ++q) {
        int o0 = st.off[q];
        int cq = st.off[q + 1] - o0;
        int sq = __shfl_sync(FULL, start, q);
        float hx = __shfl_sync(FULL, shx, q);
        float hy = __shfl_sync(FULL, shy, q);
        float hz = __shfl_sync(FULL, shz, q);
        for (int t = lane; t < cq; t += 32) {
            if (o0 + t < s.smax) {
                float4 r = __ldg(&s.rel[sq + t]);
                sm[o0 + t] = make_float4(r.x + hx, r.y + hy, r.z + hz, r.w);
            }
        }
    }
    if (lane == 0) sm[s.smax] = make_float4(kFar, kFar, kFar, __int_as_float(0));
    __syncwarp();
    return total;
}

// Global index of staged entry t (rare path).
__device__ __forceinline__ int64_t staged_global(const DevSim& s, const StencilInfo& st, int t) {
    int q = 0;
    while (q < 26 && st.off[q + 1] <= t) ++q;
    return (int64_t)s.cell_start[st.cell[q]] + (t - st.off[q]);
}

// Per-lane pair constants for the lane's species; field suffix = species of j.  Kept as
// scalars and picked with selects so that nothing is indexed at run time (no local memory).
struct LaneTab {
    float rlo0, rlo1, rhi0, rhi1, sig20, sig21, e480, e481;
    float e40, e41, vsh0, vsh1, fc0, fc1, rc0, rc1;
    float cpot;   // 0.5 for LJ force, 0 for soft sphere
    float cpe;    // 1 for LJ energy, 0 for soft sphere
    int si;
};

__device__ __forceinline__ void load_tab(const DevSim& s, int si, LaneTab& T) {
    const int k = si * 2;
    T.rlo0 = s.pt.rc2lo[k];      T.rlo1 = s.pt.rc2lo[k + 1];
    T.rhi0 = s.pt.rc2hi[k];      T.rhi1 = s.pt.rc2hi[k + 1];
    T.sig20 = s.pt.sig2[k];      T.sig21 = s.pt.sig2[k + 1];
    T.e480 = s.pt.eps48[k];      T.e481 = s.pt.eps48[k + 1];
    T.e40 = s.pt.eps4[k];        T.e41 = s.pt.eps4[k + 1];
    T.vsh0 = s.pt.vshift[k];     T.vsh1 = s.pt.vshift[k + 1];
    T.fc0 = s.pt.fcut[k];        T.fc1 = s.pt.fcut[k + 1];
    T.rc0 = (float)s.pt.drc[k];  T.rc1 = (float)s.pt.drc[k + 1];
    T.cpot = s.pt.potential == BBMD_POT_LJ ? 0.5f : 0.0f;
    T.cpe = s.pt.potential == BBMD_POT_LJ ? 1.0f : 0.0f;
    T.si = si;
}

struct Acc {
    float fx, fy, fz;
    double u, w;
};

// One pair (i, staged t).  d = x_t - x_i.
template <bool ENERGY, bool FSHIFT>
__device__ __forceinline__ void pair_mixed(const DevSim& s, const StencilInfo& st, const LaneTab& T,
                                           float4 me, float4 p, int64_t gi, int t, Acc& a) {
    float dx = p.x - me.x, dy = p.y - me.y, dz = p.z - me.z;
    float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const bool b = (__float_as_int(p.w) & 1) != 0;
    bool in = r2 < (b ? T.rlo1 : T.rlo0);
    if (!in && r2 < (b ? T.rhi1 : T.rhi0)) {
        // within the FP32 uncertainty of the cutoff: decide with the exact FP64 rule
        int64_t gj = staged_global(s, st, t);
        in = r2_exact(s, gi, gj) < s.pt.rc2[T.si * 2 + (b ? 1 : 0)];
    }
    if (in) {
        float ir2 = rcp_approx(r2);
        float s2 = (b ? T.sig21 : T.sig20) * ir2;
        float s6 = s2 * s2 * s2;
        float f = (b ? T.e481 : T.e480) * ir2 * s6 * (s6 - T.cpot);
        float ir = 0.f;
        if (FSHIFT) {
            ir = rsqrtf(r2);
            f += (b ? T.fc1 : T.fc0) * ir;
        }
        a.fx = fmaf(f, dx, a.fx);
        a.fy = fmaf(f, dy, a.fy);
        a.fz = fmaf(f, dz, a.fz);
        if (ENERGY) {
            float V = (b ? T.e41 : T.e40) * s6 * (s6 - T.cpe) - (b ? T.vsh1 : T.vsh0);
            if (FSHIFT) V -= (r2 * ir - (b ? T.rc1 : T.rc0)) * (b ? T.fc1 : T.fc0);
            a.u += (double)V;
            a.w += (double)(f * r2);
        }
    }
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Block reduction of per-warp doubles into partials[q * kMaxPartials + blockIdx.x].
__device__ void block_partials(const DevSim& s, const double* wv, int nq) {
    __shared__ double red[kWarpsPerBlock][4];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0)
        for (int q = 0; q < nq; ++q) red[w][q] = wv[q];
    __syncthreads();
    if (threadIdx.x < nq) {
        double t = 0.0;
        for (int k = 0; k < kWarpsPerBlock; ++k) t += red[k][threadIdx.x];
        s.partials[threadIdx.x * kMaxPartials + blockIdx.x] = t;
    }
}

// MODE 0: Verlet list.  MODE 1: every staged particle (no stored list).
template <int MODE, bool ENERGY, bool KE, bool FSHIFT>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_force(DevSim s) {
    extern __shared__ float4 smem[];
    __shared__ StencilInfo sinfo[kWarpsPerBlock];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float4* sm = smem + (size_t)w * (s.smax + 1);
    StencilInfo& st = sinfo[w];
    const int64_t nwarps = (int64_t)gridDim.x * kWarpsPerBlock;
    double acc_ke = 0.0, acc_u = 0.0, acc_w = 0.0;
    float hdt[2] = {0.f, 0.f};
    if (KE) {
        double dt = s.sc->dt;
        hdt[0] = (float)(0.5 * dt / s.pt.dmass[0]);
        hdt[1] = (float)(0.5 * dt / s.pt.dmass[1]);
    }
    for (int64_t c = (int64_t)blockIdx.x * kWarpsPerBlock + w; c < s.ncell; c += nwarps) {
        int total = stage_stencil(s, (int)c, sm, st, lane);
        const int i0 = s.cell_start[c];
        const int cnt = s.cell_start[c + 1] - i0;
        const int self0 = st.off[13];
        for (int ch = 0; ch * 32 < cnt; ++ch) {
            const int li = ch * 32 + lane;
            const bool act = li < cnt;
            const int64_t gi = (int64_t)i0 + li;
            float4 me = act ? sm[self0 + li] : make_float4(-kFar, -kFar, -kFar, 0.f);
            int si = __float_as_int(me.w) & 1;
            LaneTab T;
            load_tab(s, si, T);
            Acc a = {0.f, 0.f, 0.f, 0.0, 0.0};
            if (MODE == 0) {
                const int nkb = s.cellmax[i0 + ch * 32];
                const uint4* lp = reinterpret_cast<const uint4*>(s.list) + gi;
                const uint4 sent = make_uint4(s.smax | (s.smax << 16), s.smax | (s.smax << 16),
                                              s.smax | (s.smax << 16), s.smax | (s.smax << 16));
                uint4 e = (act && nkb > 0) ? __ldcs(lp) : sent;
                for (int kb = 0; kb < nkb; ++kb) {
                    uint4 en = (act && kb + 1 < nkb) ? __ldcs(lp + (int64_t)(kb + 1) * s.npad) : sent;
#define BBMD_PAIR2(W)                                                          \
    {                                                                          \
        int t0 = (W) & 0xffffu, t1 = (W) >> 16;                                \
        pair_mixed<ENERGY, FSHIFT>(s, st, T, me, sm[t0], gi, t0, a);           \
        pair_mixed<ENERGY, FSHIFT>(s, st, T, me, sm[t1], gi, t1, a);           \
    }
                    BBMD_PAIR2(e.x) BBMD_PAIR2(e.y) BBMD_PAIR2(e.z) BBMD_PAIR2(e.w)
#undef BBMD_PAIR2
                    e = en;
                }
            } else {
                const int self = self0 + li;
                for (int t = 0; t < total; ++t) {
                    float4 p = sm[t];
                    if (t == self) p = make_float4(kFar, kFar, kFar, 0.f);
                    pair_mixed<ENERGY, FSHIFT>(s, st, T, me, p, gi, t, a);
                }
            }
            float fx = -a.fx, fy = -a.fy, fz = -a.fz;
            if (act) {
                if (!(isfinite(fx) && isfinite(fy) && isfinite(fz))) set_status(s, ST_NONFINITE);
                s.F[gi] = make_float4(fx, fy, fz, ENERGY ? (float)(0.5 * a.u) : 0.f);
                if (ENERGY) s.ud[gi] = 0.5 * a.u;
            }
            if (KE) {
                float k = 0.f;
                if (act) {
                    float h = si ? hdt[1] : hdt[0];
                    float m = si ? s.pt.mass[1] : s.pt.mass[0];
                    float vx = fmaf(h, fx, i64_to_f32_fast(s.v[gi]) * pow2f(-kVelExp));
                    float vy = fmaf(h, fy, i64_to_f32_fast(s.v[s.npad + gi]) * pow2f(-kVelExp));
                    float vz = fmaf(h, fz, i64_to_f32_fast(s.v[2 * s.npad + gi]) * pow2f(-kVelExp));
                    k = 0.5f * m * fmaf(vx, vx, fmaf(vy, vy, vz * vz));
                }
                k = warp_sum_f(k);
                if (lane == 0) acc_ke += (double)k;
            }
            if (ENERGY) {
                double uu = warp_sum_d(act ? 0.5 * a.u : 0.0);
                double ww = warp_sum_d(act ? 0.5 * a.w : 0.0);
                if (lane == 0) {
                    acc_u += uu;
                    acc_w += ww;
                }
            }
        }
    }
    if (KE || ENERGY) {
        double wv[3] = {acc_ke, acc_u, acc_w};
        block_partials(s, wv, 3);
    }
}

// ------------------------------------------------------------------ list build ----

__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_list_build(DevSim s) {
    if (!s.sc->rebuild) return;
    extern __shared__ float4 smem[];
    __shared__ StencilInfo sinfo[kWarpsPerBlock];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int lcap = s.lcap8 * 8;
    const int bstride = lcap + 2;  // odd number of 32-bit words per row
    float4* sm = smem + (size_t)w * (s.smax + 1);
    uint16_t* buf = reinterpret_cast<uint16_t*>(smem + (size_t)kWarpsPerBlock * (s.smax + 1)) +
                    (size_t)w * 32 * bstride + (size_t)lane * bstride;
    StencilInfo& st = sinfo[w];
    const int64_t nwarps = (int64_t)gridDim.x * kWarpsPerBlock;
    for (int64_t c = (int64_t)blockIdx.x * kWarpsPerBlock + w; c < s.ncell; c += nwarps) {
        int total = stage_stencil(s, (int)c, sm, st, lane);
        const int i0 = s.cell_start[c];
        const int cnt = s.cell_start[c + 1] - i0;
        const int self0 = st.off[13];
        for (int ch = 0; ch * 32 < cnt; ++ch) {
            const int li = ch * 32 + lane;
            const bool act = li < cnt;
            const int64_t gi = (int64_t)i0 + li;
            const int self = self0 + li;
            float4 me = act ? sm[self] : make_float4(-kFar, -kFar, -kFar, 0.f);
            int si = __float_as_int(me.w) & 1;
            float Rlo0 = s.pt.R2lo[si * 2], Rlo1 = s.pt.R2lo[si * 2 + 1];
            float Rhi0 = s.pt.R2hi[si * 2], Rhi1 = s.pt.R2hi[si * 2 + 1];
            int len = 0;
            for (int t = 0; t < total; ++t) {
                float4 p = sm[t];
                float dx = p.x - me.x, dy = p.y - me.y, dz = p.z - me.z;
                float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                int tj = __float_as_int(p.w) & 1;
                bool in = r2 < (tj ? Rlo1 : Rlo0);
                if (!in && act && r2 < (tj ? Rhi1 : Rhi0) && t != self) {
                    int64_t gj = staged_global(s, st, t);
                    in = r2_exact(s, gi, gj) < s.pt.R2[si * 2 + tj];
                }
                if (in && act && t != self) {
                    if (len < lcap) buf[len] = (uint16_t)t;
                    ++len;
                }
            }
            if (len > lcap) {
                set_status(s, ST_LIST_OVERFLOW);
                len = lcap;
            }
            int mx = len;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(FULL, mx, o));
            const int nkb = (mx + 7) >> 3;
            for (int q = len; q < nkb * 8; ++q) buf[q] = (uint16_t)s.smax;
            if (act) {
                uint4* lp = reinterpret_cast<uint4*>(s.list) + gi;
                for (int kb = 0; kb < nkb; ++kb) {
                    const uint16_t* b = buf + kb * 8;
                    uint4 e;
                    e.x = (unsigned)b[0] | ((unsigned)b[1] << 16);
                    e.y = (unsigned)b[2] | ((unsigned)b[3] << 16);
                    e.z = (unsigned)b[4] | ((unsigned)b[5] << 16);
                    e.w = (unsigned)b[6] | ((unsigned)b[7] << 16);
                    lp[(int64_t)kb * s.npad] = e;
                }
            }
            if (lane == 0) s.cellmax[i0 + ch * 32] = (uint16_t)nkb;
            __syncwarp();
        }
    }
}

// ------------------------------------------------------------------ FP64 form ----
// Stencil staged as exact integer positions shifted into the tile's periodic image;
// distances are the exact integer differences rounded once to double (the same rule the
// list decisions use), pair arithmetic and accumulation in FP64.

struct Pos64 {
    long long x, y, z;
    int sp, pad;
};

__device__ int stage_stencil64(const DevSim& s, int c, Pos64* sm, StencilInfo& st, int lane) {
    int ax, ay, az;
    cell_coords(c, s.nc, ax, ay, az);
    int start = 0, cnt = 0, nb = 0;
    long long wx = 0, wy = 0, wz = 0;
    if (lane < 27) {
        int o[3] = {lane % 3 - 1, (lane / 3) % 3 - 1, lane / 9 - 1};
        int a[3] = {ax, ay, az};
        int b[3];
        long long wr[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            int bb = a[d] + o[d];
            wr[d] = 0;
            if (bb < 0) {
                bb += s.nc[d];
                wr[d] = -s.Lfix[d];
            } else if (bb >= s.nc[d]) {
                bb -= s.nc[d];
                wr[d] = s.Lfix[d];
            }
            b[d] = bb;
        }
        nb = (b[2] * s.nc[1] + b[1]) * s.nc[0] + b[0];
        start = s.cell_start[nb];
        cnt = s.cell_start[nb + 1] - start;
        wx = wr[0];
        wy = wr[1];
        wz = wr[2];
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += t;
    }
    int total = __shfl_sync(FULL, incl, 26);
    if (lane < 27) {
        st.off[lane] = incl - cnt;
        st.cell[lane] = nb;
    }
    if (lane == 0) st.off[27] = total;
    __syncwarp();
    if (total > s.smax) {
        if (lane == 0) set_status(s, ST_STENCIL_OVERFLOW);
        total = s.smax;
    }
    for (int q = 0; q < 27; ++q) {
        int o0 = st.off[q];
        int cq = st.off[q + 1] - o0;
        int sq = __shfl_sync(FULL, start, q);
        long long hx = __shfl_sync(FULL, wx, q);
        long long hy = __shfl_sync(FULL, wy, q);
        long long hz = __shfl_sync(FULL, wz, q);
        for (int t = lane; t < cq; t += 32) {
            if (o0 + t < s.smax) {
                int64_t j = sq + t;
                Pos64 p;
                p.x = (long long)s.x[j] + hx;
                p.y = (long long)s.x[s.npad + j] + hy;
                p.z = (long long)s.x[2 * s.npad + j] + hz;
                p.sp = s.sp[j];
                p.pad = 0;
                sm[o0 + t] = p;
            }
        }
    }
    if (lane == 0) {
        Pos64 far;
        far.x = far.y = far.z = (long long)1 << 62;
        far.sp = 0;
        far.pad = 0;
        sm[s.smax] = far;
    }
    __syncwarp();
    return total;
}

template <bool ENERGY, bool FSHIFT>
__device__ __forceinline__ void pair_fp64(const DevSim& s, int si, const Pos64& me, const Pos64& p,
                                          double& fx, double& fy, double& fz, double& u,
                                          double& w) {
    double dx = __dmul_rn(__ll2double_rn(p.x - me.x), s.sxd);
    double dy = __dmul_rn(__ll2double_rn(p.y - me.y), s.sxd);
    double dz = __dmul_rn(__ll2double_rn(p.z - me.z), s.sxd);
    double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    int k = si * 2 + p.sp;
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

template <int MODE, bool ENERGY, bool KE, bool FSHIFT>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_force64(DevSim s) {
    extern __shared__ float4 smem[];
    __shared__ StencilInfo sinfo[kWarpsPerBlock];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    Pos64* sm = reinterpret_cast<Pos64*>(smem) + (size_t)w * (s.smax + 1);
    StencilInfo& st = sinfo[w];
    const int64_t nwarps = (int64_t)gridDim.x * kWarpsPerBlock;
    double acc_ke = 0.0, acc_u = 0.0, acc_w = 0.0;
    for (int64_t c = (int64_t)blockIdx.x * kWarpsPerBlock + w; c < s.ncell; c += nwarps) {
        int total = stage_stencil64(s, (int)c, sm, st, lane);
        const int i0 = s.cell_start[c];
        const int cnt = s.cell_start[c + 1] - i0;
        const int self0 = st.off[13];
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
            int si = me.sp;
            double fx = 0, fy = 0, fz = 0, u = 0, wv = 0;
            if (MODE == 0) {
                const int nkb = s.cellmax[i0 + ch * 32];
                const uint4* lp = reinterpret_cast<const uint4*>(s.list) + gi;
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!act) break;
                    uint4 e = lp[(int64_t)kb * s.npad];
                    unsigned ws[4] = {e.x, e.y, e.z, e.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        pair_fp64<ENERGY, FSHIFT>(s, si, me, sm[ws[q] & 0xffffu], fx, fy, fz, u, wv);
                        pair_fp64<ENERGY, FSHIFT>(s, si, me, sm[ws[q] >> 16], fx, fy, fz, u, wv);
                    }
                }
            } else {
                const int self = self0 + li;
                for (int t = 0; t < total; ++t) {
                    if (t == self || !act) continue;
                    pair_fp64<ENERGY, FSHIFT>(s, si, me, sm[t], fx, fy, fz, u, wv);
                }
            }
            if (act) {
                fx = -fx;
                fy = -fy;
                fz = -fz;
                if (!(isfinite(fx) && isfinite(fy) && isfinite(fz))) set_status(s, ST_NONFINITE);
                s.Fd[gi] = fx;
                s.Fd[s.npad + gi] = fy;
                s.Fd[2 * s.npad + gi] = fz;
                s.F[gi] = make_float4((float)fx, (float)fy, (float)fz, ENERGY ? (float)(0.5 * u) : 0.f);
                if (ENERGY) s.ud[gi] = 0.5 * u;
            }
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
    if (KE || ENERGY) {
        double wv3[3] = {acc_ke, acc_u, acc_w};
        block_partials(s, wv3, 3);
    }
}

// Opt every kernel with dynamic shared memory into the device maximum once (outside any
// stream capture); the launch itself then requests only what it needs.
constexpr int kMaxDynSmem = 227 * 1024;

template <typename K>
void set_smem(K kernel, size_t /*bytes*/) {
    static bool done = false;
    if (!done) {
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
        done = true;
    }
}

template <int MODE, bool E, bool KE, bool FS>
void run_force(const DevSim& s, cudaStream_t st) {
    if (s.precision == BBMD_PREC_FP64) {
        size_t bytes = (size_t)kWarpsPerBlock * (s.smax + 1) * sizeof(Pos64);
        set_smem(k_force64<MODE, E, KE, FS>, bytes);
        k_force64<MODE, E, KE, FS><<<s.grid_cell, kWarpsPerBlock * 32, bytes, st>>>(s);
    } else {
        size_t bytes = (size_t)kWarpsPerBlock * (s.smax + 1) * sizeof(float4);
        set_smem(k_force<MODE, E, KE, FS>, bytes);
        k_force<MODE, E, KE, FS><<<s.grid_cell, kWarpsPerBlock * 32, bytes, st>>>(s);
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
    set_smem(k_force<MODE, E, KE, FS>, 0);
    set_smem(k_force64<MODE, E, KE, FS>, 0);
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

void prepare_force_kernels() {
    prep_mode<0>();
    prep_mode<1>();
    set_smem(k_list_build, 0);
}

void launch_force(const DevSim& s, cudaStream_t st, bool energy, bool ke) {
    bool fs = s.pt.shift == BBMD_SHIFT_FORCE;
    if (s.nbr_mode == BBMD_NBR_VERLET)
        run_force_mode<0>(s, st, energy, ke, fs);
    else
        run_force_mode<1>(s, st, energy, ke, fs);
}

void launch_list_build(const DevSim& s, cudaStream_t st) {
    if (s.nbr_mode != BBMD_NBR_VERLET) return;
    size_t bytes = (size_t)kWarpsPerBlock * (s.smax + 1) * sizeof(float4) +
                   (size_t)kWarpsPerBlock * 32 * (s.lcap8 * 8 + 2) * sizeof(uint16_t);
    set_smem(k_list_build, bytes);
    k_list_build<<<s.grid_cell, kWarpsPerBlock * 32, bytes, st>>>(s);
}

}  // namespace bbmd
