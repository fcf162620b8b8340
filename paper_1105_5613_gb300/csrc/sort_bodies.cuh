// Device bodies of the cell binning and spatial reorder (Sec. 2.2: O(N) cell search over
// cubic cells; the paper's per-cell linked lists become a counting sort into contiguous
// cell segments).  Each body runs for one system given (system, CTA index within it, CTA
// count of it) and is gated on sc->rebuild.  The kernels of k_sort.cu wrap them for one
// system or a replica batch; the persistent batch kernel calls them phase after phase.
// Included inside an anonymous namespace.
#pragma once

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 8;
constexpr int kScanChunk = kScanThreads * kScanItems;

__host__ __device__ __forceinline__ int scan_chunks(const DevSim& s) {
    return (int)((s.ncell + kScanChunk - 1) / kScanChunk);
}

__device__ __forceinline__ void zero_body(const DevSim& s, int lb, int lg) {
    if (!s.sc->rebuild) return;
    if (lb == 0 && threadIdx.x == 0) {  // the list build of this rebuild sets them afresh
        s.sc->list_short = 0;
        s.sc->max_len = 0;
    }
    for (int64_t c = lb * (int64_t)blockDim.x + threadIdx.x; c <= s.ncell;
         c += (int64_t)lg * blockDim.x) {
        s.count[c] = 0;
        s.cursor[c] = 0;
    }
}

__device__ __forceinline__ void bin_body(const DevSim& s, int lb, int lg) {
    if (!s.sc->rebuild) return;
    for (int64_t i = lb * (int64_t)blockDim.x + threadIdx.x; i < s.n;
         i += (int64_t)lg * blockDim.x) {
        int ax = cell_axis((long long)s.x[i], s.D[0], s.nc[0]);
        int ay = cell_axis((long long)s.x[s.npad + i], s.D[1], s.nc[1]);
        int az = cell_axis((long long)s.x[2 * s.npad + i], s.D[2], s.nc[2]);
        int c = (az * s.nc[1] + ay) * s.nc[0] + ax;
        s.key[i] = c;
        atomicAdd(&s.count[c], 1);
    }
}

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ int block_scan_excl(int v, int& total) {
    __shared__ int wsum[kScanThreads / 32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        int x = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
        int xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += t;
        }
        wsum[lane] = xi - x;
        if (lane == (int)(blockDim.x >> 5) - 1) total = xi;
    }
    __syncthreads();
    int r = wsum[w] + incl - v;
    __syncthreads();
    return r;
}

// pass 1: per-chunk sums of count[0 .. ncell)
__device__ __forceinline__ void scan_reduce_body(const DevSim& s, int lb, int lg) {
    if (!s.sc->rebuild) return;
    const int nchunks = scan_chunks(s);
    __shared__ int red[kScanThreads / 32];
    for (int ch = lb; ch < nchunks; ch += lg) {
        int64_t base = (int64_t)ch * kScanChunk + (int64_t)threadIdx.x * kScanItems;
        int acc = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            int64_t c = base + k;
            if (c < s.ncell) acc += s.count[c];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x < 32) {
            int x = threadIdx.x < (kScanThreads / 32) ? red[threadIdx.x] : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (threadIdx.x == 0) s.scan_part[ch] = x;
        }
        __syncthreads();
    }
}

// pass 2: exclusive scan of the chunk sums (one block)
__device__ __forceinline__ void scan_top_body(const DevSim& s, int lb, int lg) {
    if (!s.sc->rebuild) return;
    const int nchunks = scan_chunks(s);
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nchunks; base += kScanThreads) {
        int idx = base + threadIdx.x;
        int v = idx < nchunks ? s.scan_part[idx] : 0;
        int total = 0;
        __shared__ int tot;
        int ex = block_scan_excl(v, tot);
        total = tot;
        if (idx < nchunks) s.scan_part[idx] = ex + carry;
        __syncthreads();
        if (threadIdx.x == 0) carry += total;
        __syncthreads();
    }
}

// pass 3: per-chunk exclusive scan plus chunk offset -> cell_start
__device__ __forceinline__ void scan_down_body(const DevSim& s, int lb, int lg) {
    if (!s.sc->rebuild) return;
    const int nchunks = scan_chunks(s);
    for (int ch = lb; ch < nchunks; ch += lg) {
        int64_t base = (int64_t)ch * kScanChunk + (int64_t)threadIdx.x * kScanItems;
        int vals[kScanItems];
        int acc = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            int64_t c = base + k;
            vals[k] = c < s.ncell ? s.count[c] : 0;
            acc += vals[k];
        }
        __shared__ int tot;
        int ex = block_scan_excl(acc, tot) + s.scan_part[ch];
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            int64_t c = base + k;
            if (c < s.ncell) s.cell_start[c] = ex;
            ex += vals[k];
        }
    }
    if (lb == 0 && threadIdx.x == 0) s.cell_start[s.ncell] = (int32_t)s.n;
}

// The whole exclusive scan count -> cell_start by one CTA of any multiple-of-32 size (the
// persistent batch kernel: a replica has few cells).  Integer sums: the same cell_start
// as the three-pass scan.
__device__ __forceinline__ void scan_cta_body(const DevSim& s, int lb, int lg) {
    if (!s.sc->rebuild || lb != 0) return;
    __shared__ int carry;
    __shared__ int tot;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int64_t per = (int64_t)blockDim.x * kScanItems;
    for (int64_t base0 = 0; base0 < s.ncell; base0 += per) {
        const int64_t base = base0 + (int64_t)threadIdx.x * kScanItems;
        int vals[kScanItems];
        int acc = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            const int64_t c = base + k;
            vals[k] = c < s.ncell ? s.count[c] : 0;
            acc += vals[k];
        }
        int ex = block_scan_excl(acc, tot) + carry;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            const int64_t c = base + k;
            if (c < s.ncell) s.cell_start[c] = ex;
            ex += vals[k];
        }
        __syncthreads();  // every thread has read carry
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) s.cell_start[s.ncell] = (int32_t)s.n;
}

__device__ __forceinline__ void scatter_body(const DevSim& s, int lb, int lg) {
    if (!s.sc->rebuild) return;
    for (int64_t i = lb * (int64_t)blockDim.x + threadIdx.x; i < s.n;
         i += (int64_t)lg * blockDim.x) {
        int c = s.key[i];
        int slot = s.cell_start[c] + atomicAdd(&s.cursor[c], 1);
        s.perm_tmp[slot] = (int32_t)i;
    }
}

// Order each cell's particles by (species, id): rank = number of smaller keys in the cell.
// Species A first lets the force kernel form warps of one species; the order is canonical
// (it depends only on positions, species and ids).
__device__ __forceinline__ long long cell_key(const DevSim& s, int p) {
    return ((long long)s.sp[p] << 32) | (long long)(unsigned)s.id[p];
}

__device__ __forceinline__ void cellsort_body(const DevSim& s, int lb, int lg) {
    if (!s.sc->rebuild) return;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)lg * (blockDim.x >> 5);
    for (int64_t c = (lb * (int64_t)blockDim.x + threadIdx.x) >> 5; c < s.ncell;
         c += nwarps) {
        int start = s.cell_start[c];
        int cnt = s.cell_start[c + 1] - start;
        if (cnt <= 32) {
            int pe = lane < cnt ? s.perm_tmp[start + lane] : 0;
            long long key = lane < cnt ? cell_key(s, pe) : 0x7fffffffffffffffll;
            int rank = 0;
            for (int f = 0; f < cnt; ++f) {
                long long other = __shfl_sync(0xffffffffu, key, f);
                rank += other < key;
            }
            if (lane < cnt) s.perm[start + rank] = pe;
        } else {
            for (int e = lane; e < cnt; e += 32) {
                int pe = s.perm_tmp[start + e];
                long long key = cell_key(s, pe);
                int rank = 0;
                for (int f = 0; f < cnt; ++f) rank += cell_key(s, s.perm_tmp[start + f]) < key;
                s.perm[start + rank] = pe;
            }
        }
    }
}

__device__ __forceinline__ void gather_body(const DevSim& s, int lb, int lg) {
    if (!s.sc->rebuild) return;
    for (int64_t k = lb * (int64_t)blockDim.x + threadIdx.x; k < s.n;
         k += (int64_t)lg * blockDim.x) {
        int64_t o = s.perm[k];
        // all loads of the particle first (the stores could alias them for the compiler)
        const int c = s.key[o];
        uint64_t xv[3];
        int64_t vv[3];
        int32_t iv[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            xv[d] = s.x[d * s.npad + o];
            vv[d] = s.v[d * s.npad + o];
            iv[d] = s.img[d * s.npad + o];
        }
        const int32_t idv = s.id[o];
        const uint8_t spc = s.sp[o];
        int ax, ay, az;
        cell_coords(c, s.nc, ax, ay, az);
        int a3[3] = {ax, ay, az};
        float r[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            s.x2[d * s.npad + k] = xv[d];
            s.v2[d * s.npad + k] = vv[d];
            s.img2[d * s.npad + k] = iv[d];
            long long rel = (long long)xv[d] - frame_axis(a3[d], s.D[d]);
            r[d] = i64_to_f32(rel) * s.sx;
        }
        s.id2[k] = idv;
        s.sp2[k] = spc;
        s.relb[k] = make_float4(r[0], r[1], r[2], __int_as_float((c << 1) | spc));
        s.rel[k] = make_float4(r[0], r[1], r[2], (float)spc);
    }
}

__device__ __forceinline__ void copyback_body(const DevSim& s, int lb, int lg) {
    if (!s.sc->rebuild) return;
    for (int64_t k = lb * (int64_t)blockDim.x + threadIdx.x; k < s.n;
         k += (int64_t)lg * blockDim.x) {
        uint64_t xv[3];
        int64_t vv[3];
        int32_t iv[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            xv[d] = s.x2[d * s.npad + k];
            vv[d] = s.v2[d * s.npad + k];
            iv[d] = s.img2[d * s.npad + k];
        }
        const int32_t idv = s.id2[k];
        const uint8_t spc = s.sp2[k];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            s.x[d * s.npad + k] = xv[d];
            s.v[d * s.npad + k] = vv[d];
            s.img[d * s.npad + k] = iv[d];
        }
        s.id[k] = idv;
        s.sp[k] = spc;
    }
}

