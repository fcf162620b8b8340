// Radial distribution function (Sec. 4, the g(r) of the glass study): partial ordered-pair
// histograms n_ab(q), q = floor(r / dr), r from the exact r^2 rule.
//
// Pairs are found on a coarse grid of cells of side >= rmax (one CTA per coarse cell, the
// 27 neighbour cells streamed through shared memory) or, when the box holds fewer than
// three such cells per axis, by all pairs.  Distances are formed from the exact integer
// displacement rounded once to FP32; a pair whose r / dr lies within 5e-4 of a bin edge is
// binned again with the FP64 rule, so every count equals the FP64 definition.
#include "bbmd_internal.cuh"

namespace bbmd {

namespace {

constexpr int kT = 256;
constexpr int kChunk = 256;
constexpr float kEdgeTol = 5e-4f;

struct GrArgs {
    int nbins;
    float inv_dr, rmax2_hi;
    double dr;
    int ncg[3];
    long long Dg[3];
    int ncells;
    int32_t *gkey, *gidx, *gcount, *gstart, *gcursor;
};

__device__ __forceinline__ int bin_exact(const DevSim& s, const GrArgs& g, long long dx,
                                         long long dy, long long dz) {
    double a = __dmul_rn(__ll2double_rn(dx), s.sxd);
    double b = __dmul_rn(__ll2double_rn(dy), s.sxd);
    double c = __dmul_rn(__ll2double_rn(dz), s.sxd);
    double r2 = __dadd_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)), __dmul_rn(c, c));
    double q = floor(__ddiv_rn(__dsqrt_rn(r2), g.dr));
    return q < (double)g.nbins ? (int)q : -1;
}

// Bin of one pair from its exact integer displacement (-1: outside the range).
__device__ __forceinline__ int pair_bin(const DevSim& s, const GrArgs& g, long long dx, long long dy,
                                       long long dz) {
    float fx = i64_to_f32(dx) * s.sx, fy = i64_to_f32(dy) * s.sx, fz = i64_to_f32(dz) * s.sx;
    float r2 = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
    if (!(r2 < g.rmax2_hi)) return -1;
    float qf = sqrtf(r2) * g.inv_dr;
    float fl = floorf(qf);
    float fr = qf - fl;
    if (fr < kEdgeTol || fr > 1.0f - kEdgeTol || fl >= (float)g.nbins - 1.0f)
        return bin_exact(s, g, dx, dy, dz);
    return (int)fl;
}

__global__ void k_gr_zero(GrArgs g) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= g.ncells; c += gridDim.x * blockDim.x) {
        g.gcount[c] = 0;
        g.gcursor[c] = 0;
    }
}

__global__ void k_gr_key(DevSim s, GrArgs g) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int a[3];
        for (int d = 0; d < 3; ++d) a[d] = cell_axis((long long)s.x[d * s.npad + i], g.Dg[d], g.ncg[d]);
        int c = (a[2] * g.ncg[1] + a[1]) * g.ncg[0] + a[0];
        g.gkey[i] = c;
        atomicAdd(&g.gcount[c], 1);
    }
}

__global__ void k_gr_scan(GrArgs g) {
    // one block: exclusive scan of gcount into gstart
    __shared__ int carry;
    __shared__ int ws[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < g.ncells; base += blockDim.x) {
        int idx = base + threadIdx.x;
        int v = idx < g.ncells ? g.gcount[idx] : 0;
        int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        int incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) ws[w] = incl;
        __syncthreads();
        if (w == 0) {
            int x = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0;
            int xi = x;
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(0xffffffffu, xi, o);
                if (lane >= o) xi += t;
            }
            ws[lane] = xi - x;
        }
        __syncthreads();
        int ex = ws[w] + incl - v;
        if (idx < g.ncells) g.gstart[idx] = carry + ex;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += ex + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) g.gstart[g.ncells] = carry;
}

__global__ void k_gr_scatter(DevSim s, GrArgs g) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int c = g.gkey[i];
        g.gidx[g.gstart[c] + atomicAdd(&g.gcursor[c], 1)] = (int32_t)i;
    }
}

struct JEnt {
    long long x, y, z;
    int sp, gi;
};

__device__ void flush_hist(unsigned* hist, int nb4, unsigned long long* counts) {
    __syncthreads();
    for (int q = threadIdx.x; q < nb4; q += blockDim.x)
        if (hist[q]) atomicAdd(&counts[q], (unsigned long long)hist[q]);
    __syncthreads();
    for (int q = threadIdx.x; q < nb4; q += blockDim.x) hist[q] = 0;
    __syncthreads();
}

__global__ void __launch_bounds__(kT) k_gr_cells(DevSim s, GrArgs g, unsigned long long* counts) {
    extern __shared__ unsigned char gsm[];
    JEnt* stg = reinterpret_cast<JEnt*>(gsm);
    unsigned* hist = reinterpret_cast<unsigned*>(stg + kChunk);
    const int nb4 = 4 * g.nbins;
    for (int q = threadIdx.x; q < nb4; q += blockDim.x) hist[q] = 0;
    __syncthreads();
    for (int c = blockIdx.x; c < g.ncells; c += gridDim.x) {
        int a[3] = {c % g.ncg[0], (c / g.ncg[0]) % g.ncg[1], c / (g.ncg[0] * g.ncg[1])};
        int cs = g.gstart[c], ce = g.gstart[c + 1];
        for (int ib = cs; ib < ce; ib += kT) {
            int li = ib + threadIdx.x;
            bool act = li < ce;
            int64_t gi = act ? g.gidx[li] : 0;
            long long xi = act ? (long long)s.x[gi] : 0, yi = act ? (long long)s.x[s.npad + gi] : 0,
                      zi = act ? (long long)s.x[2 * s.npad + gi] : 0;
            int si = act ? s.sp[gi] : 0;
            for (int q = 0; q < 27; ++q) {
                int o[3] = {q % 3 - 1, (q / 3) % 3 - 1, q / 9 - 1};
                int b[3];
                long long wr[3];
                for (int d = 0; d < 3; ++d) {
                    int bb = a[d] + o[d];
                    wr[d] = 0;
                    if (bb < 0) {
                        bb += g.ncg[d];
                        wr[d] = -s.Lfix[d];
                    } else if (bb >= g.ncg[d]) {
                        bb -= g.ncg[d];
                        wr[d] = s.Lfix[d];
                    }
                    b[d] = bb;
                }
                int nb = (b[2] * g.ncg[1] + b[1]) * g.ncg[0] + b[0];
                int js = g.gstart[nb], je = g.gstart[nb + 1];
                for (int jb = js; jb < je; jb += kChunk) {
                    int cntc = min(kChunk, je - jb);
                    __syncthreads();
                    for (int t = threadIdx.x; t < cntc; t += blockDim.x) {
                        int gj = g.gidx[jb + t];
                        JEnt e;
                        e.x = (long long)s.x[gj] + wr[0];
                        e.y = (long long)s.x[s.npad + gj] + wr[1];
                        e.z = (long long)s.x[2 * s.npad + gj] + wr[2];
                        e.sp = s.sp[gj];
                        e.gi = gj;
                        stg[t] = e;
                    }
                    __syncthreads();
                    if (act) {
                        for (int t = 0; t < cntc; ++t) {
                            JEnt e = stg[t];
                            if (e.gi == (int)gi) continue;
                            int bin = pair_bin(s, g, e.x - xi, e.y - yi, e.z - zi);
                            if (bin >= 0) atomicAdd(&hist[(si * 2 + e.sp) * g.nbins + bin], 1u);
                        }
                    }
                }
            }
        }
    }
    flush_hist(hist, nb4, counts);
}

// All pairs (small boxes): block b takes i in [b*kT, b*kT + kT), j streamed in chunks.
__global__ void __launch_bounds__(kT) k_gr_all(DevSim s, GrArgs g, unsigned long long* counts) {
    extern __shared__ unsigned char gsm[];
    JEnt* stg = reinterpret_cast<JEnt*>(gsm);
    unsigned* hist = reinterpret_cast<unsigned*>(stg + kChunk);
    const int nb4 = 4 * g.nbins;
    for (int q = threadIdx.x; q < nb4; q += blockDim.x) hist[q] = 0;
    __syncthreads();
    for (int64_t ib = (int64_t)blockIdx.x * kT; ib < s.n; ib += (int64_t)gridDim.x * kT) {
        int64_t gi = ib + threadIdx.x;
        bool act = gi < s.n;
        long long xi = act ? (long long)s.x[gi] : 0, yi = act ? (long long)s.x[s.npad + gi] : 0,
                  zi = act ? (long long)s.x[2 * s.npad + gi] : 0;
        int si = act ? s.sp[gi] : 0;
        for (int64_t jb = 0; jb < s.n; jb += kChunk) {
            int cntc = (int)min((int64_t)kChunk, s.n - jb);
            __syncthreads();
            for (int t = threadIdx.x; t < cntc; t += blockDim.x) {
                int64_t gj = jb + t;
                JEnt e;
                e.x = (long long)s.x[gj];
                e.y = (long long)s.x[s.npad + gj];
                e.z = (long long)s.x[2 * s.npad + gj];
                e.sp = s.sp[gj];
                e.gi = (int)gj;
                stg[t] = e;
            }
            __syncthreads();
            if (act) {
                for (int t = 0; t < cntc; ++t) {
                    JEnt e = stg[t];
                    if (e.gi == (int)gi) continue;
                    long long dx = min_image(e.x - xi, s.Lfix[0]);
                    long long dy = min_image(e.y - yi, s.Lfix[1]);
                    long long dz = min_image(e.z - zi, s.Lfix[2]);
                    int bin = pair_bin(s, g, dx, dy, dz);
                    if (bin >= 0) atomicAdd(&hist[(si * 2 + e.sp) * g.nbins + bin], 1u);
                }
            }
        }
        // keep the 32-bit shared counters far from overflow
        flush_hist(hist, nb4, counts);
    }
    flush_hist(hist, nb4, counts);
}

}  // namespace

// scratch_i32: 2 n + 3 (ncells + 1) ints.  Returns 0, or -1 if scratch is too small.
int launch_gr(const DevSim& s, cudaStream_t st, int nbins, double rmax,
              unsigned long long* counts_dev, int32_t* scratch_i32, float4* /*scratch_f4*/,
              int64_t scratch_n) {
    GrArgs g;
    g.nbins = nbins;
    g.dr = rmax / (double)nbins;
    g.inv_dr = (float)(1.0 / g.dr);
    g.rmax2_hi = (float)(rmax * rmax * 1.001);
    bool cells = true;
    g.ncells = 1;
    for (int d = 0; d < 3; ++d) {
        double L = ldexp((double)s.Lfix[d], -s.kexp);
        int m = (int)floor(L / rmax);
        if (m < 3) cells = false;
        g.ncg[d] = m < 1 ? 1 : m;
        g.Dg[d] = s.Lfix[d] / g.ncg[d];
        g.ncells *= g.ncg[d];
    }
    size_t smem = kChunk * sizeof(JEnt) + (size_t)4 * nbins * sizeof(unsigned);
    cudaMemsetAsync(counts_dev, 0, sizeof(unsigned long long) * 4 * nbins, st);
    if (!cells) {
        cudaFuncSetAttribute(k_gr_all, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int nblk = (int)((s.n + kT - 1) / kT);
        k_gr_all<<<nblk, kT, smem, st>>>(s, g, counts_dev);
        return 0;
    }
    if (scratch_n < 2 * s.n + 3 * ((int64_t)g.ncells + 1)) return -1;
    g.gkey = scratch_i32;
    g.gidx = scratch_i32 + s.n;
    g.gcount = scratch_i32 + 2 * s.n;
    g.gstart = g.gcount + (g.ncells + 1);
    g.gcursor = g.gstart + (g.ncells + 1);
    k_gr_zero<<<256, 256, 0, st>>>(g);
    k_gr_key<<<s.grid_part, 256, 0, st>>>(s, g);
    k_gr_scan<<<1, 1024, 0, st>>>(g);
    k_gr_scatter<<<s.grid_part, 256, 0, st>>>(s, g);
    cudaFuncSetAttribute(k_gr_cells, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nblk = g.ncells < 65535 * 4 ? g.ncells : 65535 * 4;
    k_gr_cells<<<nblk, kT, smem, st>>>(s, g, counts_dev);
    return 0;
}

}  // namespace bbmd
