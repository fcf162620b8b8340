// Velocity-Verlet time marching (Sec. 2.3.2) with an optional Nose-Hoover thermostat
// (the paper's canonical runs, Sec. 3, do not name the thermostat; a single friction
// variable is used), device reductions ("a few limited global collective operations",
// Sec. 2.3.1, become fixed-order FP64 block sums) and state transfer.
//
// Step pipeline (one launch each, all on the handle's stream):
//   integrate : v <- s (v + pend h F) + h F ; x <- x + v dt ; wrap ; frame copy ; flag
//   [rebuild chain + list build, gated on the flag]
//   force     : F(x) (+ kinetic-energy partials of v + h F when thermostatted)
//   finalize  : K = sum of partials; NH half at the end of this step and at the start of
//               the next; the product of both velocity scales is applied by the next
//               integrate, so each particle's velocity is touched once per step.
// The second half kick of the last step of a call is applied by finish.
//
// Mixed precision keeps positions and velocities in 64-bit fixed point and forms every
// increment in FP32; no FP64 arithmetic runs per particle per step (GB300 issues FP64 at
// a small fraction of the FP32 rate).
#include <algorithm>

#include "bbmd_internal.cuh"

namespace bbmd {

namespace {

constexpr int kThreads = 256;
constexpr unsigned FULL = 0xffffffffu;

#include "step_bodies.cuh"

// Start of a call.  If the previous call's closing half kick and Nose-Hoover scale are
// still pending (the velocities were not finished: sc->pending), they are carried into
// the first velocity update of this call, which applies s_end (v + h F) and this call's
// scale and first half kick in one increment; the host carries only when dt is unchanged
// (the pending kick and the first kick use the same h).
__global__ void k_begin(DevSim s, int64_t nsteps, double dt, int kind, double T0, double T1,
                        double tau) {
    DevScalars* sc = s.sc;
    const bool carry = sc->pending != 0;
    const double s_carry = carry ? sc->s_end : 1.0;
    sc->dt = dt;
    sc->hdt[0] = (float)(0.5 * dt / s.pt.dmass[0]);
    sc->hdt[1] = (float)(0.5 * dt / s.pt.dmass[1]);
    sc->n_in_call = (int)nsteps;
    sc->step_in_call = 0;
    sc->kind = kind;
    sc->T_start = T0;
    sc->T_end = T1;
    sc->tau = tau;
    sc->pending = carry ? 1 : 0;
    sc->g = (double)(3 * s.n - 3);
    if (kind == BBMD_THERMO_NH) {
        double Kout;
        sc->s_next = nh_half(sc, sc->K, ramp_T(sc, 0), dt, &Kout) * s_carry;
        sc->K = Kout;
        sc->T_last = ramp_T(sc, 0);
    } else {
        sc->s_next = s_carry;
    }
    sc->s_end = 1.0;
}

// Four CTAs per SM (64 registers; the compiler would take 92 and fit two): the kernel is
// bound by HBM, and more resident warps keep more of its loads in flight.
template <bool FP64>
__global__ void __launch_bounds__(kThreads, 4) k_integrate(DevSim s) {
    integrate_body<FP64>(s, (int)blockIdx.x, (int)gridDim.x);
}

BBMD_ONE_AND_MANY(kThreads, k_celltop, celltop_body)
BBMD_ONE_AND_MANY(kThreads, k_check, check_body)

template <bool FP64>
__global__ void __launch_bounds__(kThreads, 4) k_integrate_many(ManySims m) {
    __shared__ DevSim sh;
    int lb, lg;
    load_replica(m, sh, lb, lg);
    integrate_body<FP64>(sh, lb, lg);
}

__global__ void __launch_bounds__(256) k_finalize(DevSim s, int ke) { finalize_body(s, ke); }

__global__ void __launch_bounds__(256) k_finalize_many(ManySims m, int ke) {
    __shared__ DevSim sh;
    int lb, lg;
    load_replica(m, sh, lb, lg);
    finalize_body(sh, ke);
}

// The finished velocity of particle i: the pending closing half kick and Nose-Hoover
// scale of the last call applied, v + round(s_end (v + h F) - v) (the arithmetic of the
// closing update), or the stored velocity when nothing is pending.
template <bool FP64>
__device__ __forceinline__ void finished_velocity(const DevSim& s, int64_t i, long long vo[3]) {
    const DevScalars* sc = s.sc;
#pragma unroll
    for (int d = 0; d < 3; ++d) vo[d] = s.v[d * s.npad + i];
    if (!sc->pending) return;
    const double dt = sc->dt;
    const double se = sc->s_end;
    const int spc = s.sp[i];
    if (!FP64) {
        const float4 F = s.F[i];
        const float Fv[3] = {F.x, F.y, F.z};
        const float h = 0.5f * (float)dt / s.pt.mass[spc];
        const float sm1 = (float)(se - 1.0);
        const float sf = (float)se;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float vf = i64_to_f32_fast(vo[d]) * pow2f(-kVelExp);
            const float dv = fmaf(sm1, vf, sf * h * Fv[d]);
            vo[d] += f32_to_i64(dv * pow2f(kVelExp));
        }
    } else {
        const double h = 0.5 * dt / s.pt.dmass[spc];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double vd = __ll2double_rn(vo[d]) * 0x1p-52;
            const double dv = (se - 1.0) * vd + se * h * s.Fd[d * s.npad + i];
            vo[d] += __double2ll_rn(dv * 0x1p52);
        }
    }
}

// Apply the pending closing update to the stored velocities (nothing when none is pending;
// k_finish_done then marks the velocities finished).
template <bool FP64>
__global__ void __launch_bounds__(kThreads) k_finish(DevSim s) {
    if (!s.sc->pending) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        long long vo[3];
        finished_velocity<FP64>(s, i, vo);
#pragma unroll
        for (int d = 0; d < 3; ++d) s.v[d * s.npad + i] = vo[d];
    }
}

__global__ void k_finish_done(DevSim s) { s.sc->pending = 0; }

// Kinetic energy and momentum (FP64) of the finished velocities (the stored ones with any
// pending closing update applied on the fly, as the finish kernel would) -> partials 0..3.
template <bool FP64>
__global__ void __launch_bounds__(kThreads) k_state_sums(DevSim s) {
    double k = 0, px = 0, py = 0, pz = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double m = s.pt.dmass[s.sp[i]];
        long long vo[3];
        finished_velocity<FP64>(s, i, vo);
        double vx = __ll2double_rn(vo[0]) * 0x1p-52;
        double vy = __ll2double_rn(vo[1]) * 0x1p-52;
        double vz = __ll2double_rn(vo[2]) * 0x1p-52;
        k += 0.5 * m * (vx * vx + vy * vy + vz * vz);
        px += m * vx;
        py += m * vy;
        pz += m * vz;
    }
    __shared__ double red[4][kThreads];
    red[0][threadIdx.x] = k;
    red[1][threadIdx.x] = px;
    red[2][threadIdx.x] = py;
    red[3][threadIdx.x] = pz;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4) s.partials[threadIdx.x * kMaxPartials + blockIdx.x] = red[threadIdx.x][0];
}

__global__ void __launch_bounds__(256) k_reduce_partials(DevSim s, int nb, int nq, double* out,
                                                        int set_K) {
    __shared__ double r[8];
    sum_partials(s, nb, nq, r);
    if (threadIdx.x == 0) {
        for (int q = 0; q < nq; ++q) out[q] = r[q];
        if (set_K) s.sc->K = r[0];
    }
}

// ------------------------------------------------------------------ initialisers ----

__device__ __forceinline__ unsigned long long splitmix_mix(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ unsigned long long draw(unsigned long long seed, int stream,
                                                   unsigned long long c) {
    unsigned long long ctr = ((unsigned long long)stream << 40) | c;
    return splitmix_mix(seed + (ctr + 1ull) * 0x9E3779B97F4A7C15ull);
}

__device__ __forceinline__ long long quantize_dev(double x, int k, long long L) {
    long long q = __double2ll_rn(ldexp(x, k));
    q %= L;
    if (q < 0) q += L;
    return q;
}

// FCC site i (4 m^3 sites): ((ix, iy, iz) + basis_b + 1/4) L/m, then, when jitter > 0,
// coordinate d moved by jitter (2u - 1) with u the uniform draw 3i + d of stream 5 (the
// same IEEE operations as the Python generator: no fused multiply-add).
__global__ void __launch_bounds__(kThreads) k_init_fcc(DevSim s, int m, double Lx, double Ly,
                                                      double Lz, double jitter,
                                                      unsigned long long seed) {
    const double bx[4] = {0.0, 0.5, 0.5, 0.0}, by[4] = {0.0, 0.5, 0.0, 0.5},
                 bz[4] = {0.0, 0.0, 0.5, 0.5};
    double ax = Lx / m, ay = Ly / m, az = Lz / m;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int b = (int)(i & 3);
        int64_t cidx = i >> 2;
        int64_t ix = cidx % m, iy = (cidx / m) % m, iz = cidx / ((int64_t)m * m);
        double p3[3] = {((double)ix + bx[b] + 0.25) * ax, ((double)iy + by[b] + 0.25) * ay,
                        ((double)iz + bz[b] + 0.25) * az};
        if (jitter > 0.0) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const unsigned long long z = draw(seed, 5, 3ull * (unsigned long long)i + d);
                const double u = (double)(z >> 11) * 0x1p-53;
                p3[d] = __dadd_rn(p3[d], __dmul_rn(jitter, __dsub_rn(__dmul_rn(2.0, u), 1.0)));
            }
        }
        const double px = p3[0], py = p3[1], pz = p3[2];
        s.x[i] = (uint64_t)quantize_dev(px, s.kexp, s.Lfix[0]);
        s.x[s.npad + i] = (uint64_t)quantize_dev(py, s.kexp, s.Lfix[1]);
        s.x[2 * s.npad + i] = (uint64_t)quantize_dev(pz, s.kexp, s.Lfix[2]);
    }
}

// Gaussian draws scaled by sqrt(T/m) into tmp[3][n] (id order) + momentum partials.
__global__ void __launch_bounds__(kThreads) k_mb_draw(DevSim s, double T, unsigned long long seed,
                                                     double* tmp) {
    double px = 0, py = 0, pz = 0, mt = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double m = s.pt.dmass[s.sp[i]];
        double sc = sqrt(T / m);
        double v3[3];
        for (int d = 0; d < 3; ++d) {
            unsigned long long mm = 3ull * (unsigned long long)i + d;
            unsigned long long z1 = draw(seed, 2, 2ull * mm), z2 = draw(seed, 2, 2ull * mm + 1ull);
            double u1 = (double)((z1 >> 11) + 1ull) * 0x1p-53;
            double u2 = (double)(z2 >> 11) * 0x1p-53;
            double g = sqrt(-2.0 * log(u1)) * cos(2.0 * 3.141592653589793 * u2);
            v3[d] = g * sc;
            tmp[d * s.n + i] = v3[d];
        }
        px += m * v3[0];
        py += m * v3[1];
        pz += m * v3[2];
        mt += m;
    }
    __shared__ double red[4][kThreads];
    red[0][threadIdx.x] = px;
    red[1][threadIdx.x] = py;
    red[2][threadIdx.x] = pz;
    red[3][threadIdx.x] = mt;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4) s.partials[threadIdx.x * kMaxPartials + blockIdx.x] = red[threadIdx.x][0];
}

// Remove the mean momentum; kinetic-energy partials of the result.
__global__ void __launch_bounds__(kThreads) k_mb_shift(DevSim s, double* tmp, const double* P) {
    double vx0 = P[0] / P[3], vy0 = P[1] / P[3], vz0 = P[2] / P[3];
    double k = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double m = s.pt.dmass[s.sp[i]];
        double a = tmp[i] - vx0, b = tmp[s.n + i] - vy0, c = tmp[2 * s.n + i] - vz0;
        tmp[i] = a;
        tmp[s.n + i] = b;
        tmp[2 * s.n + i] = c;
        k += m * a * a + m * b * b + m * c * c;
    }
    __shared__ double red[kThreads];
    red[threadIdx.x] = k;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) s.partials[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(kThreads) k_mb_scale(DevSim s, const double* tmp,
                                                      const double* KE2, double T) {
    double ke = 0.5 * KE2[0];
    double f = 1.0;
    if (s.n > 1 && T > 0.0) f = sqrt(T / (2.0 * ke / (double)(3 * s.n - 3)));
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        for (int d = 0; d < 3; ++d) {
            double v = T > 0.0 ? tmp[d * s.n + i] * f : 0.0;
            s.v[d * s.npad + i] = __double2ll_rn(v * 0x1p52);
        }
    }
}

// ------------------------------------------------------------ steepest descent ----

__global__ void __launch_bounds__(kThreads) k_maxf(DevSim s) {
    float m = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float4 F = s.F[i];
        m = fmaxf(m, F.x * F.x + F.y * F.y + F.z * F.z);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(FULL, m, o));
    __shared__ float red[kThreads / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int k = 0; k < kThreads / 32; ++k) t = fmaxf(t, red[k]);
        s.partials[blockIdx.x] = (double)t;
    }
}

__global__ void k_maxf_final(DevSim s, int nb) {
    if (threadIdx.x != 0) return;
    double m = 0.0;
    for (int b = 0; b < nb; ++b) m = fmax(m, s.partials[b]);
    s.sc->maxf = sqrt(m);
}

template <bool FP64>
__global__ void __launch_bounds__(kThreads) k_sd_move(DevSim s, double hmax, double dmax) {
    double fm = s.sc->maxf;
    double h = hmax;
    if (fm > 0.0 && dmax / fm < h) h = dmax / fm;
    bool need = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float4 rb = s.relb[i];
        int wb = __float_as_int(rb.w);
        int c = wb >> 1;
        int a3[3] = {c % s.nc[0], (c / s.nc[0]) % s.nc[1], c / (s.nc[0] * s.nc[1])};
        float4 F = s.F[i];
        float Fv[3] = {F.x, F.y, F.z};
        float r[3];
        for (int d = 0; d < 3; ++d) {
            int64_t idx = d * s.npad + i;
            double f = FP64 ? s.Fd[idx] : (double)Fv[d];
            long long x = (long long)s.x[idx] + __double2ll_rn(ldexp(h * f, s.kexp));
            if (x >= s.Lfix[d]) {
                x -= s.Lfix[d];
                s.img[idx] += 1;
            } else if (x < 0) {
                x += s.Lfix[d];
                s.img[idx] -= 1;
            }
            s.x[idx] = (uint64_t)x;
            r[d] = i64_to_f32(min_image(x - frame_axis(a3[d], s.D[d]), s.Lfix[d])) * s.sx;
        }
        s.rel[i] = make_float4(r[0], r[1], r[2], (float)(wb & 1));
        float ex = r[0] - rb.x, ey = r[1] - rb.y, ez = r[2] - rb.z;
        if (fmaf(ex, ex, fmaf(ey, ey, ez * ez)) > s.disp2) need = true;
    }
    if (__any_sync(FULL, need) && (threadIdx.x & 31) == 0) s.sc->rebuild = 1;
}

__global__ void k_clear_rebuild(DevSim s) {
    if (s.sc->rebuild) {
        s.sc->n_rebuilds += 1;
        s.sc->rebuild = 0;
    }
}

// --------------------------------------------------------------- state transfer ----

__global__ void __launch_bounds__(kThreads) k_unpack_state(DevSim s, double* pos, double* vel,
                                                          int32_t* img) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < s.n;
         k += (int64_t)gridDim.x * blockDim.x) {
        int64_t id = s.id[k];
        for (int d = 0; d < 3; ++d) {
            int64_t idx = d * s.npad + k;
            if (pos) pos[3 * id + d] = ldexp(__ll2double_rn((long long)s.x[idx]), -s.kexp);
            if (vel) vel[3 * id + d] = __ll2double_rn(s.v[idx]) * 0x1p-52;
            if (img) img[3 * id + d] = s.img[idx];
        }
    }
}

// Species by id (scatter through the current order) into sp2.
__global__ void __launch_bounds__(kThreads) k_species_by_id(DevSim s) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < s.n;
         k += (int64_t)gridDim.x * blockDim.x)
        s.sp2[s.id[k]] = s.sp[k];
}

// Uploaded state check: one CTA-wide vote per CTA, a flag written only when some value is
// not finite.
__global__ void __launch_bounds__(kThreads) k_check_finite(DevSim s, const double* a, int64_t m) {
    int bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        bad |= !isfinite(a[i]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) s.sc->bad_input = 1;
}

__global__ void __launch_bounds__(kThreads) k_pack_state(DevSim s, const double* pos,
                                                        const double* vel, const int32_t* img) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < s.n;
         k += (int64_t)gridDim.x * blockDim.x) {
        s.id[k] = (int32_t)k;
        s.sp[k] = s.sp2[k];
        for (int d = 0; d < 3; ++d) {
            int64_t idx = d * s.npad + k;
            if (pos) s.x[idx] = (uint64_t)quantize_dev(pos[3 * k + d], s.kexp, s.Lfix[d]);
            if (vel) s.v[idx] = __double2ll_rn(vel[3 * k + d] * 0x1p52);
            s.img[idx] = img ? img[3 * k + d] : 0;
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_unpack_forces(DevSim s, double* F, double* u) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < s.n;
         k += (int64_t)gridDim.x * blockDim.x) {
        int64_t id = s.id[k];
        if (s.precision == BBMD_PREC_FP64) {
            for (int d = 0; d < 3; ++d) F[3 * id + d] = s.Fd[d * s.npad + k];
        } else {
            float4 f = s.F[k];
            F[3 * id] = f.x;
            F[3 * id + 1] = f.y;
            F[3 * id + 2] = f.z;
        }
        if (u) u[id] = s.ud[k];
    }
}

// Forces of the particles ids[0..m) (slot_of: sorted position of each id).
__global__ void __launch_bounds__(kThreads) k_forces_of_ids(DevSim s, const int32_t* slot_of,
                                                           const int64_t* ids, int64_t m,
                                                           double* F, double* u) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = slot_of[ids[t]];
        if (s.precision == BBMD_PREC_FP64) {
            for (int d = 0; d < 3; ++d) F[3 * t + d] = s.Fd[d * s.npad + k];
        } else {
            const float4 f = s.F[k];
            F[3 * t] = f.x;
            F[3 * t + 1] = f.y;
            F[3 * t + 2] = f.z;
        }
        if (u) u[t] = s.ud[k];
    }
}

__global__ void __launch_bounds__(kThreads) k_unpack_cells(DevSim s, int64_t* cell) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < s.n;
         k += (int64_t)gridDim.x * blockDim.x)
        cell[s.id[k]] = __float_as_int(s.relb[k].w) >> 1;
}

// Global slot of staged offset t in the region of the block that holds cell c (the cells
// around the block in the force kernel's staging order).
__device__ int64_t stencil_slot(const DevSim& s, int c, int t) {
    int ax, ay, az;
    cell_coords(c, s.nc, ax, ay, az);
    const int bxy = block_xy_of(s.block_z), bzc = block_zc_of(s.block_z), rxy = bxy + 2;
    const int a0[3] = {ax - ax % bxy, ay - ay % bxy, az - az % bzc};
    int acc = 0;
    for (int q = 0; q < s.region_cells; ++q) {
        const int r[3] = {q % rxy, (q / rxy) % rxy, q / (rxy * rxy)};
        int b[3];
        for (int d = 0; d < 3; ++d) {
            int bb = a0[d] - 1 + r[d];
            if (bb < 0) bb += s.nc[d];
            else if (bb >= s.nc[d]) bb -= s.nc[d];
            b[d] = bb;
        }
        int nb = (b[2] * s.nc[1] + b[1]) * s.nc[0] + b[0];
        int st = s.cell_start[nb], cnt = s.cell_start[nb + 1] - st;
        if (t < acc + cnt) return (int64_t)st + (t - acc);
        acc += cnt;
    }
    return -1;
}

__device__ __forceinline__ int list_len(const DevSim& s, int64_t k, int nkb) {
    int len = 0;
    const uint4* lp = reinterpret_cast<const uint4*>(s.list) + k;
    for (int kb = 0; kb < nkb; ++kb) {
        uint4 e = lp[(int64_t)kb * s.npad];
        unsigned w4[4] = {e.x, e.y, e.z, e.w};
        for (int q = 0; q < 4; ++q) {
            len += (int)((w4[q] & 0xffffu) != (unsigned)s.smax);
            len += (int)((w4[q] >> 16) != (unsigned)s.smax);
        }
    }
    return len;
}

__device__ __forceinline__ int tile_nkb(const DevSim& s, int64_t k) { return s.rows[k]; }

__global__ void __launch_bounds__(kThreads) k_slot_of(DevSim s, int32_t* slot_of) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < s.n;
         k += (int64_t)gridDim.x * blockDim.x)
        slot_of[s.id[k]] = (int32_t)k;
}

__global__ void __launch_bounds__(kThreads) k_list_counts(DevSim s, const int32_t* sel, int64_t m,
                                                         int64_t* counts) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t k = sel ? sel[t] : t;
        int64_t o = sel ? t : s.id[k];
        counts[o] = list_len(s, k, tile_nkb(s, k));
    }
}

__global__ void __launch_bounds__(kThreads) k_list_ids(DevSim s, const int32_t* sel, int64_t m,
                                                      const int64_t* off, int64_t* nbr) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t k = sel ? sel[t] : t;
        int64_t o = sel ? t : s.id[k];
        int c = __float_as_int(s.relb[k].w) >> 1;
        int nkb = tile_nkb(s, k);
        int64_t base = off[o];
        int64_t len = 0;
        const uint4* lp = reinterpret_cast<const uint4*>(s.list) + k;
        for (int kb = 0; kb < nkb; ++kb) {
            uint4 e = lp[(int64_t)kb * s.npad];
            unsigned w4[4] = {e.x, e.y, e.z, e.w};
            for (int q = 0; q < 8; ++q) {
                unsigned tt = (q & 1) ? (w4[q >> 1] >> 16) : (w4[q >> 1] & 0xffffu);
                if (tt == (unsigned)s.smax) continue;
                int64_t slot = stencil_slot(s, c, (int)tt);
                nbr[base + len++] = slot >= 0 ? s.id[slot] : -1;
            }
        }
        // ascending ids (insertion sort of one short list)
        for (int64_t a = 1; a < len; ++a) {
            int64_t v = nbr[base + a];
            int64_t b = a - 1;
            while (b >= 0 && nbr[base + b] > v) {
                nbr[base + b + 1] = nbr[base + b];
                --b;
            }
            nbr[base + b + 1] = v;
        }
    }
}

// ------------------------------------------------------------ MSD and F_s ----

__global__ void __launch_bounds__(kThreads) k_set_ref(DevSim s, double* ref, double Lx, double Ly,
                                                     double Lz) {
    const double L[3] = {Lx, Ly, Lz};
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < s.n;
         k += (int64_t)gridDim.x * blockDim.x) {
        int64_t id = s.id[k];
        for (int d = 0; d < 3; ++d) {
            int64_t idx = d * s.npad + k;
            ref[d * s.n + id] =
                ldexp(__ll2double_rn((long long)s.x[idx]), -s.kexp) + L[d] * (double)s.img[idx];
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_msd_fs(DevSim s, const double* ref, double kv,
                                                    double Lx, double Ly, double Lz) {
    const double L[3] = {Lx, Ly, Lz};
    double acc[6] = {0, 0, 0, 0, 0, 0};  // msdA, msdB, fsA, fsB, nA, nB
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < s.n;
         k += (int64_t)gridDim.x * blockDim.x) {
        int64_t id = s.id[k];
        int a = s.sp[k];
        double d2 = 0.0, c = 0.0;
        for (int d = 0; d < 3; ++d) {
            int64_t idx = d * s.npad + k;
            double u = ldexp(__ll2double_rn((long long)s.x[idx]), -s.kexp) + L[d] * (double)s.img[idx];
            double du = u - ref[d * s.n + id];
            d2 += du * du;
            c += cos(kv * du);
        }
        acc[a] += d2;
        acc[2 + a] += c / 3.0;
        acc[4 + a] += 1.0;
    }
    __shared__ double red[6][kThreads];
    for (int q = 0; q < 6; ++q) red[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int q = 0; q < 6; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 6) s.partials[threadIdx.x * kMaxPartials + blockIdx.x] = red[threadIdx.x][0];
}

}  // namespace

void launch_begin(const DevSim& s, cudaStream_t st, int64_t nsteps, double dt,
                  const bbmd_thermostat* th) {
    int kind = th ? th->kind : BBMD_THERMO_NVE;
    double T0 = th ? th->T_start : 0.0, T1 = th ? th->T_end : 0.0, tau = th ? th->tau : 1.0;
    k_begin<<<1, 1, 0, st>>>(s, nsteps, dt, kind, T0, T1, tau);
}

void launch_integrate(const DevSim& s, cudaStream_t st) {
    if (s.precision == BBMD_PREC_FP64)
        k_integrate<true><<<s.grid_part, kThreads, 0, st>>>(s);
    else
        k_integrate<false><<<s.grid_part, kThreads, 0, st>>>(s);
}

void launch_check(const DevSim& s, cudaStream_t st) {
    const int g = (int)std::min<int64_t>(s.grid_part, (s.ncell + kThreads - 1) / kThreads);
    k_celltop<<<s.grid_part, kThreads, 0, st>>>(s);
    k_check<<<g > 0 ? g : 1, kThreads, 0, st>>>(s);
}

void launch_check_many(const ManySims& part, int total, cudaStream_t st) {
    k_celltop_many<<<total, kThreads, 0, st>>>(part);
    k_check_many<<<total, kThreads, 0, st>>>(part);
}

void launch_finalize(const DevSim& s, cudaStream_t st, bool ke) {
    k_finalize<<<1, 256, 0, st>>>(s, ke ? 1 : 0);
}

void launch_integrate_many(const ManySims& part, int total, bool fp64, cudaStream_t st) {
    if (fp64)
        k_integrate_many<true><<<total, kThreads, 0, st>>>(part);
    else
        k_integrate_many<false><<<total, kThreads, 0, st>>>(part);
}

void launch_finalize_many(const ManySims& one, int nrep, bool ke, cudaStream_t st) {
    k_finalize_many<<<nrep, 256, 0, st>>>(one, ke ? 1 : 0);
}

void launch_finish(const DevSim& s, cudaStream_t st) {
    if (s.precision == BBMD_PREC_FP64)
        k_finish<true><<<s.grid_part, kThreads, 0, st>>>(s);
    else
        k_finish<false><<<s.grid_part, kThreads, 0, st>>>(s);
    k_finish_done<<<1, 1, 0, st>>>(s);
}

void launch_state_sums(const DevSim& s, cudaStream_t st) {
    if (s.precision == BBMD_PREC_FP64)
        k_state_sums<true><<<s.grid_part, kThreads, 0, st>>>(s);
    else
        k_state_sums<false><<<s.grid_part, kThreads, 0, st>>>(s);
}

void launch_reduce_partials(const DevSim& s, cudaStream_t st, int nq, double* out_dev) {
    // nq > 0: partials written by a per-particle kernel (grid_part blocks);
    // nq < 0: by a per-cell kernel (grid_cell blocks), |nq| quantities.
    int nb = nq > 0 ? s.grid_part : s.grid_cell;
    int q = nq > 0 ? nq : -nq;
    k_reduce_partials<<<1, 256, 0, st>>>(s, nb, q, out_dev, 0);
}

void launch_init_fcc(const DevSim& s, cudaStream_t st, int m, double jitter, uint64_t seed) {
    k_init_fcc<<<s.grid_part, kThreads, 0, st>>>(s, m, ldexp((double)s.Lfix[0], -s.kexp),
                                                 ldexp((double)s.Lfix[1], -s.kexp),
                                                 ldexp((double)s.Lfix[2], -s.kexp), jitter,
                                                 (unsigned long long)seed);
}

void launch_init_mb(const DevSim& s, cudaStream_t st, double T0, uint64_t seed, double* tmp3) {
    // tmp3: 3n doubles of scratch followed by 8 doubles for the sums
    double* sums = tmp3 + 3 * s.n;
    k_mb_draw<<<s.grid_part, kThreads, 0, st>>>(s, T0, seed, tmp3);
    k_reduce_partials<<<1, 256, 0, st>>>(s, s.grid_part, 4, sums, 0);
    k_mb_shift<<<s.grid_part, kThreads, 0, st>>>(s, tmp3, sums);
    k_reduce_partials<<<1, 256, 0, st>>>(s, s.grid_part, 1, sums + 4, 0);
    k_mb_scale<<<s.grid_part, kThreads, 0, st>>>(s, tmp3, sums + 4, T0);
}

void launch_sd_step(const DevSim& s, cudaStream_t st, double hmax, double dmax) {
    k_maxf<<<s.grid_part, kThreads, 0, st>>>(s);
    k_maxf_final<<<1, 32, 0, st>>>(s, s.grid_part);
    if (s.precision == BBMD_PREC_FP64)
        k_sd_move<true><<<s.grid_part, kThreads, 0, st>>>(s, hmax, dmax);
    else
        k_sd_move<false><<<s.grid_part, kThreads, 0, st>>>(s, hmax, dmax);
}

void launch_clear_rebuild(const DevSim& s, cudaStream_t st) { k_clear_rebuild<<<1, 1, 0, st>>>(s); }

void launch_set_ref(const DevSim& s, cudaStream_t st, double* ref) {
    k_set_ref<<<s.grid_part, kThreads, 0, st>>>(s, ref, ldexp((double)s.Lfix[0], -s.kexp),
                                                ldexp((double)s.Lfix[1], -s.kexp),
                                                ldexp((double)s.Lfix[2], -s.kexp));
}

void launch_msd_fs(const DevSim& s, cudaStream_t st, const double* ref, double kvec,
                   double* out_dev) {
    k_msd_fs<<<s.grid_part, kThreads, 0, st>>>(s, ref, kvec, ldexp((double)s.Lfix[0], -s.kexp),
                                               ldexp((double)s.Lfix[1], -s.kexp),
                                               ldexp((double)s.Lfix[2], -s.kexp));
    k_reduce_partials<<<1, 256, 0, st>>>(s, s.grid_part, 6, out_dev, 0);
}

void launch_unpack_state(const DevSim& s, cudaStream_t st, double* pos, double* vel,
                         int32_t* img) {
    k_unpack_state<<<s.grid_part, kThreads, 0, st>>>(s, pos, vel, img);
}

void launch_pack_state(const DevSim& s, cudaStream_t st, const double* pos, const double* vel,
                       const int32_t* img, bool species_from_current) {
    if (species_from_current) k_species_by_id<<<s.grid_part, kThreads, 0, st>>>(s);
    k_pack_state<<<s.grid_part, kThreads, 0, st>>>(s, pos, vel, img);
}

void launch_check_finite(const DevSim& s, cudaStream_t st, const double* a, int64_t m) {
    k_check_finite<<<s.grid_part, kThreads, 0, st>>>(s, a, m);
}

void launch_unpack_forces(const DevSim& s, cudaStream_t st, double* F, double* u) {
    k_unpack_forces<<<s.grid_part, kThreads, 0, st>>>(s, F, u);
}

void launch_forces_of_ids(const DevSim& s, cudaStream_t st, const int32_t* slot_of,
                          const int64_t* ids, int64_t m, double* F, double* u) {
    const int g = (int)std::min<int64_t>(s.grid_part, (m + kThreads - 1) / kThreads);
    k_forces_of_ids<<<g > 0 ? g : 1, kThreads, 0, st>>>(s, slot_of, ids, m, F, u);
}

void launch_unpack_cells(const DevSim& s, cudaStream_t st, int64_t* cell) {
    k_unpack_cells<<<s.grid_part, kThreads, 0, st>>>(s, cell);
}

void launch_slot_of(const DevSim& s, cudaStream_t st, int32_t* slot_of) {
    k_slot_of<<<s.grid_part, kThreads, 0, st>>>(s, slot_of);
}

void launch_list_counts(const DevSim& s, cudaStream_t st, const int32_t* sel, int64_t m,
                        int64_t* counts) {
    k_list_counts<<<s.grid_part, kThreads, 0, st>>>(s, sel, m, counts);
}

void launch_list_ids(const DevSim& s, cudaStream_t st, const int32_t* sel, int64_t m,
                     const int64_t* offsets, int64_t* nbr) {
    k_list_ids<<<s.grid_part, kThreads, 0, st>>>(s, sel, m, offsets, nbr);
}

}  // namespace bbmd
