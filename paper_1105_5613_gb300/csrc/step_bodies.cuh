// Device bodies of the per-step kernels of the integrator: the velocity-Verlet update
// with the Nose-Hoover halves (Sec. 2.3.2; the canonical runs of Sec. 3), the rebuild
// trigger and the fixed-order reduction that closes a step.  Each body runs for one
// system given (system, CTA index within it, CTA count of it); the kernels of
// k_integrate.cu wrap them for one system or a replica batch, and the persistent batch
// kernel calls them phase after phase.  Included inside an anonymous namespace.
#pragma once

constexpr int kStepThreads = 256;
constexpr unsigned kStepFull = 0xffffffffu;

__device__ __forceinline__ double nh_half(DevScalars* sc, double K, double T, double dt,
                                          double* Kout) {
    double g = sc->g;
    double Q = g * T * sc->tau * sc->tau;
    sc->xi += 0.25 * dt * (2.0 * K - g * T) / Q;
    double s = exp(-sc->xi * 0.5 * dt);
    K = K * s * s;
    sc->eta += sc->xi * 0.5 * dt;
    sc->xi += 0.25 * dt * (2.0 * K - g * T) / Q;
    *Kout = K;
    return s;
}

__device__ __forceinline__ double ramp_T(const DevScalars* sc, int k) {
    return sc->T_start + (sc->T_end - sc->T_start) * (double)k / (double)sc->n_in_call;
}

template <bool FP64>
__device__ __forceinline__ void integrate_body(const DevSim& s, int lb, int lg) {
    const DevScalars* sc = s.sc;
    const double dt = sc->dt;
    const double snext = sc->s_next;
    const int pend = sc->pending;
    const float dtf = (float)dt;
    const float sm1 = (float)(snext - 1.0);
    const float coef = pend ? (float)snext + 1.0f : 1.0f;
    const float hf[2] = {0.5f * dtf / s.pt.mass[0], 0.5f * dtf / s.pt.mass[1]};
    const float vscale = pow2f(-kVelExp);
    const float vtofix = pow2f(kVelExp);
    const float dtx = dtf * pow2f(s.kexp > 126 ? 126 : s.kexp);  // k <= 61 in practice
    const int lane = threadIdx.x & 31;
    const float half_thr =
        0.5f * (s.nbr_mode == BBMD_NBR_VERLET ? fminf(s.disp_thr, s.disp_far) : s.disp_far);
    bool near = false;
    for (int64_t base = lb * (int64_t)blockDim.x + (threadIdx.x & ~31); base < s.n;
         base += (int64_t)lg * blockDim.x) {
        const int64_t i = base + lane;
        int c = -1;  // build cell (-1: no particle)
        float disp = 0.f;
        if (i < s.n) {
        // every input of the particle is loaded before the first store (the stores could
        // alias the later loads as far as the compiler knows)
        const float4 rb = s.relb[i];
        long long vin[3], xin[3];
        float Fv[3] = {0.f, 0.f, 0.f};
        if (!FP64) {
            const float4 F = s.F[i];
            Fv[0] = F.x;
            Fv[1] = F.y;
            Fv[2] = F.z;
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            vin[d] = s.v[d * s.npad + i];
            xin[d] = (long long)s.x[d * s.npad + i];
        }
        int wb = __float_as_int(rb.w);
        int spc = wb & 1;
        c = wb >> 1;
        int a3[3];
        a3[0] = c % s.nc[0];
        a3[1] = (c / s.nc[0]) % s.nc[1];
        a3[2] = c / (s.nc[0] * s.nc[1]);
        float r[3];
        float vmax = 0.f;
        if (!FP64) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                int64_t idx = d * s.npad + i;
                long long v = vin[d];
                float vf = i64_to_f32_fast(v) * vscale;
                float dv = fmaf(sm1, vf, coef * hf[spc] * Fv[d]);
                v += f32_to_i64(dv * vtofix);
                s.v[idx] = v;
                float vn = i64_to_f32_fast(v) * vscale;
                vmax = fmaxf(vmax, fabsf(vn));
                long long x = xin[d] + f32_to_i64(vn * dtx);
                if (x >= s.Lfix[d]) {
                    x -= s.Lfix[d];
                    s.img[idx] += 1;
                } else if (x < 0) {
                    x += s.Lfix[d];
                    s.img[idx] -= 1;
                }
                s.x[idx] = (uint64_t)x;
                long long rel = min_image(x - frame_axis(a3[d], s.D[d]), s.Lfix[d]);
                r[d] = i64_to_f32(rel) * s.sx;
            }
        } else {
            const double hd = 0.5 * dt / s.pt.dmass[spc];
            const double cd = pend ? snext + 1.0 : 1.0;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                int64_t idx = d * s.npad + i;
                long long v = vin[d];
                double vd = __ll2double_rn(v) * 0x1p-52;
                double dv = (snext - 1.0) * vd + cd * hd * s.Fd[idx];
                v += __double2ll_rn(dv * 0x1p52);
                s.v[idx] = v;
                double vn = __ll2double_rn(v) * 0x1p-52;
                vmax = fmaxf(vmax, (float)fabs(vn));
                long long x = xin[d] + __double2ll_rn(ldexp(vn * dt, s.kexp));
                if (x >= s.Lfix[d]) {
                    x -= s.Lfix[d];
                    s.img[idx] += 1;
                } else if (x < 0) {
                    x += s.Lfix[d];
                    s.img[idx] -= 1;
                }
                s.x[idx] = (uint64_t)x;
                long long rel = min_image(x - frame_axis(a3[d], s.D[d]), s.Lfix[d]);
                r[d] = i64_to_f32(rel) * s.sx;
            }
        }
        if (!(vmax < 1000.f)) set_status(s, ST_VEL_RANGE);
        s.rel[i] = make_float4(r[0], r[1], r[2], (float)spc);
        // displacement since the last build (read by the rebuild trigger)
        const float ex = r[0] - rb.x, ey = r[1] - rb.y, ez = r[2] - rb.z;
        disp = sqrtf(fmaf(ex, ex, fmaf(ey, ey, ez * ez)));
        }
        if (c >= 0) s.disp[i] = disp;
        near = near || disp > half_thr;
    }
    // the trigger's passes run only in steps where some particle got near the threshold
    if (__any_sync(kStepFull, near) && lane == 0) s.sc->near = 1;
}

// Rebuild trigger.  Since the last build, a pair (i, j) has come closer by at most
// d_i + d_j, the sum of the two displacements.  Two kinds of pairs could start to interact
// unseen:
//   (1) Verlet mode: a pair of the same or of neighbouring build cells that the list left
//       out.  Its distance at the build was at least rc_ab + skin, so it interacts only
//       after closing more than the skin.
//   (2) Both modes: a pair whose build cells are two apart along some axis (and at most
//       two apart along every axis: pairs three or more cells apart would have to close
//       more than 2 D - rc).  One whole cell of side D lies between them, so they were
//       more than D_min apart (the smallest side over the axes) and interact only after
//       closing more than D_min - rc_max, where rc_max is the largest cutoff.  The cell
//       grid makes D_min >= rc_max + skin, but by little when the cells just fit.
// Rule (1) compares, for every build cell, its two largest displacements, and its largest
// with the largest of each of its 26 neighbours, with the skin.  Rule (2) compares its
// largest with the largest of each cell of the 5 x 5 x 5 block around it (and with its own
// second largest) with D_min - rc_max.  Both thresholds carry a relative margin of 1e-4
// against the FP32 rounding of the displacements.  Cell mode evaluates every pair of the
// 27 build cells at every step, so only rule (2) applies there.  Pass 1 finds the two
// largest displacements of every cell (a warp per cell, the particles of a cell being
// contiguous); pass 2 applies the rules from the cells whose largest displacement exceeds
// half of the smaller threshold.  Both passes run only in steps where some displacement
// exceeds that half.
__device__ __forceinline__ void top2_insert(float v, float& a, float& b) {
    if (v > a) {
        b = a;
        a = v;
    } else if (v > b) {
        b = v;
    }
}

__device__ __forceinline__ void celltop_body(const DevSim& s, int lb, int lg) {
    if (!s.sc->near) return;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)lg * (blockDim.x >> 5);
    for (int64_t c = (lb * (int64_t)blockDim.x + threadIdx.x) >> 5; c < s.ncell; c += nwarps) {
        const int st = s.cell_start[c], en = s.cell_start[c + 1];
        float a = 0.f, b = 0.f;
        for (int k = st + lane; k < en; k += 32) top2_insert(s.disp[k], a, b);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oa = __shfl_xor_sync(kStepFull, a, o);
            const float ob = __shfl_xor_sync(kStepFull, b, o);
            top2_insert(oa, a, b);
            top2_insert(ob, a, b);
        }
        if (lane == 0) s.mtop[c] = make_float2(a, b);
    }
}

// Periodic cell index for a in [-2, n + 2) (every axis has at least 3 cells).
__device__ __forceinline__ int wrap_cell(int a, int n) {
    return a < 0 ? a + n : (a >= n ? a - n : a);
}

__device__ __forceinline__ void check_body(const DevSim& s, int lb, int lg) {
    DevScalars* sc = s.sc;
    if (!sc->near) return;
    const bool verlet = s.nbr_mode == BBMD_NBR_VERLET;
    const float thr1 = s.disp_thr, thr2 = s.disp_far;
    const float start = 0.5f * (verlet ? fminf(thr1, thr2) : thr2);
    bool need = false;
    for (int64_t c = lb * (int64_t)blockDim.x + threadIdx.x; c < s.ncell;
         c += (int64_t)lg * blockDim.x) {
        const float2 m = s.mtop[c];
        if (m.x <= start) continue;
        float m27 = m.y, m125 = m.y;  // the cell's own second largest
        int a[3];
        cell_coords((int)c, s.nc, a[0], a[1], a[2]);
        for (int dz = -2; dz <= 2; ++dz) {
            const int z = wrap_cell(a[2] + dz, s.nc[2]);
            for (int dy = -2; dy <= 2; ++dy) {
                const int y = wrap_cell(a[1] + dy, s.nc[1]);
                for (int dx = -2; dx <= 2; ++dx) {
                    if ((dx | dy | dz) == 0) continue;
                    const int x = wrap_cell(a[0] + dx, s.nc[0]);
                    const float v = s.mtop[(z * s.nc[1] + y) * s.nc[0] + x].x;
                    m125 = fmaxf(m125, v);
                    if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1 && dz >= -1 && dz <= 1)
                        m27 = fmaxf(m27, v);
                }
            }
        }
        if ((verlet && m.x + m27 > thr1) || m.x + m125 > thr2) need = true;
    }
    if (need) sc->rebuild = 1;
}

// Sum partials[q][0 .. nb) for q < nq (at most 8) in a fixed order: a strided sum per
// thread, a butterfly over each warp's lanes, then the warps in order (one CTA of at most
// 256 threads).
__device__ void sum_partials(const DevSim& s, int nb, int nq, double* out) {
    __shared__ double red[8][kStepThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int q = 0; q < nq; ++q) {
        double t = 0.0;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) t += s.partials[q * kMaxPartials + b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kStepFull, t, o);
        if (lane == 0) red[q][w] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int q = 0; q < nq; ++q) {
            double t = 0.0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[q][k];
            out[q] = t;
        }
    __syncthreads();
}

// The force kernel's grid_cell blocks wrote the kinetic-energy partials.
__device__ __forceinline__ void finalize_body(const DevSim& s, int ke) {
    __shared__ double K[1];
    DevScalars* sc = s.sc;
    if (ke) sum_partials(s, s.grid_cell, 1, K);
    if (threadIdx.x != 0) return;
    const int k = sc->step_in_call;
    const double dt = sc->dt;
    if (sc->kind == BBMD_THERMO_NH) {
        double Kb = K[0];
        sc->kin_last = Kb;
        double T = ramp_T(sc, k), K1, K2;
        double sb = nh_half(sc, Kb, T, dt, &K1);
        sc->T_last = T;
        if (k + 1 < sc->n_in_call) {
            double sa = nh_half(sc, K1, ramp_T(sc, k + 1), dt, &K2);
            sc->s_next = sb * sa;
            sc->K = K2;
        } else {
            sc->s_end = sb;
            sc->K = K1;
        }
    } else {
        sc->s_next = 1.0;
        sc->s_end = 1.0;
    }
    sc->pending = 1;
    sc->step_in_call = k + 1;
    sc->step += 1;
    sc->near = 0;
    if (sc->rebuild) {
        sc->n_rebuilds += 1;
        sc->rebuild = 0;
    }
}

