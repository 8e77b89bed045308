// Steps a5-a6: drift, kinetic energy and local energy per walker, FP64.
// With a Jastrow factor (Psi = e^J Det_up Det_dn, Sec. II.C) the drift gains
// grad_e J and the kinetic term lap_e J + |grad_e J|^2 + 2 grad_e J . b_e (b_e
// the determinants' drift), J is added to log|Psi| (FP64 pair sums, one warp
// per electron).
//
//   drift_{e,l} = sum_k (D^-1)_{ek} d_l phi_k(r_e)     (Eq. 2 with the
//   lap_e       = sum_k (D^-1)_{ek} lap phi_k(r_e)      Sec. II.C vector products;
//   T           = -1/2 sum_e lap_e                       Psi is linear in column e)
//   V_en = -sum_{e,a} Z_a / |r_e - Q_a|,  V_ee = sum_{i<j} 1 / |r_i - r_j|,
//   V_nn = sum_{a<b} Z_a Z_b / |Q_a - Q_b| (load time),  E_L = T + V (Eq. 4)
//
// One CTA per walker; one warp per electron row for the dot products (rows
// of D^-1 and of C2..C5 are contiguous); warp-shuffle reductions.
//
// FP64 path: everything in FP64.  Mixed path (C2..C4 in FP32): the drift
// dots in FP32 (D^-1 truncated to float by integer operations), the
// Laplacian dot in FP64, and the Coulomb sums in float-float on the FP32
// pipes: differences of float-pair positions, r^2 as a float pair, 1/r from
// the FP32 reciprocal square root refined by one Newton step (relative error
// ~2^-43), sums kept as float pairs.
#include <math.h>

#include <type_traits>

#include "ff_math.cuh"
#include "qmc_internal.cuh"

namespace qmc {

constexpr int kEnThreads = 256;
constexpr int kEnWarps = kEnThreads / 32;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// x rounded toward zero to a float by integer operations (|x| in the normal
// float range or 0; used where a 2^-23 relative error is acceptable)
__device__ __forceinline__ float f32_trunc(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7ff) - 1023 + 127;
    if (ex <= 0) return 0.f;
    const unsigned int f = (unsigned int)(b >> 32 & 0x80000000u) | ((unsigned int)min(ex, 254) << 23) |
                           (unsigned int)((b >> 29) & 0x7fffffu);
    return __uint_as_float(f);
}

// 1/r for the float-pair difference (dx, dy, dz)
__device__ __forceinline__ float2 ff_inv_r(float2 dx, float2 dy, float2 dz)
{
    const float2 r2 = ff::add(ff::add(ff::mul(dx, dx), ff::mul(dy, dy)), ff::mul(dz, dz));
    const float y0 = rsqrtf(r2.x);
    const float y0s = __fmul_rn(y0, y0);
    const float2 t = make_float2(y0s, fmaf(y0, y0, -y0s));      // y0^2 exactly
    const float2 e = ff::sub(make_float2(1.f, 0.f), ff::mul(r2, t));   // 1 - r2 y0^2, small
    return ff::renorm(y0, 0.5f * y0 * e.x);                      // Newton step y0 (1 + e/2)
}

// Coulomb sums of one walker in float-float (mixed path); rs: 3N positions,
// qs: 3 n_atom nuclear positions, zs: charges, all staged in shared memory.
__device__ __forceinline__ void coulomb_ff(const SysDev &s, const float2 *rs, const float2 *qs, const float *zs,
                                           double &ven, double &vee)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int N = s.n_elec;
    float2 en = make_float2(0.f, 0.f), ee = make_float2(0.f, 0.f);
    for (int e = wid; e < N; e += kEnWarps) {
        const float2 rx = rs[3 * e], ry = rs[3 * e + 1], rz = rs[3 * e + 2];
        for (int a = lane; a < s.n_atom; a += 32) {
            const float2 y = ff_inv_r(ff::sub(rx, qs[3 * a]), ff::sub(ry, qs[3 * a + 1]), ff::sub(rz, qs[3 * a + 2]));
            en = ff::add(en, ff::mulf(y, zs[a]));
        }
        for (int j = e + 1 + lane; j < N; j += 32)
            ee = ff::add(ee, ff_inv_r(ff::sub(rx, rs[3 * j]), ff::sub(ry, rs[3 * j + 1]), ff::sub(rz, rs[3 * j + 2])));
    }
    ven = -ff::val(en);
    vee = ff::val(ee);
}

// Drift and Laplacian of the determinants for electron e (one warp; results
// on every lane): b_l = sum_k (D^-1)_{ek} C_{1+l}[e][k], lap = sum_k (D^-1)_{ek} C5[e][k].
template <bool kMixed, typename TG>
__device__ __forceinline__ void dets_drift_lap(const SysDev &s, const double *__restrict__ Dinv,
                                               const TG *__restrict__ Cg, const CView &cv, int w, int e, int lane,
                                               size_t msz, double &b0, double &b1, double &b2, double &b3)
{
    const int spin = e >= s.n_up;
    const int ei = spin ? e - s.n_up : e;
    const int ns = spin ? s.n_dn : s.n_up;
    const size_t nu2 = (size_t)s.n_up * s.n_up;
    const size_t soff = spin ? nu2 : 0;
    const size_t nss = (size_t)ns * ns;
    const double *drow = Dinv + (size_t)w * msz + soff + (size_t)ei * ns;
    const TG *grow = Cg + (size_t)w * cv.g_wstride + (spin ? cv.g_ncomp * nu2 : 0) + (size_t)ei * ns;
    const double *lrow = cv.l + (size_t)w * cv.l_wstride + (spin ? cv.l_ncomp * nu2 : 0) +
                         (size_t)cv.l_comp * nss + (size_t)ei * ns;
    b0 = b1 = b2 = b3 = 0.0;
    if constexpr (kMixed) {
        float f0 = 0.f, f1 = 0.f, f2 = 0.f;
        for (int k = lane; k < ns; k += 32) {
            const double d = drow[k];
            const float df = f32_trunc(d);
            f0 = fmaf(df, grow[k], f0);
            f1 = fmaf(df, grow[nss + k], f1);
            f2 = fmaf(df, grow[2 * nss + k], f2);
            b3 = fma(d, lrow[k], b3);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            f0 += __shfl_xor_sync(0xffffffffu, f0, off);
            f1 += __shfl_xor_sync(0xffffffffu, f1, off);
            f2 += __shfl_xor_sync(0xffffffffu, f2, off);
        }
        b0 = f0; b1 = f1; b2 = f2;
    } else {
        for (int k = lane; k < ns; k += 32) {
            const double d = drow[k];
            b0 = fma(d, (double)grow[k], b0);
            b1 = fma(d, (double)grow[nss + k], b1);
            b2 = fma(d, (double)grow[2 * nss + k], b2);
            b3 = fma(d, lrow[k], b3);
        }
        b0 = warp_sum(b0); b1 = warp_sum(b1); b2 = warp_sum(b2);
    }
    b3 = warp_sum(b3);
}

// The Jastrow factor's part for electron e (one warp, FP64; results on every
// lane): g = grad_e J, L = lap_e J, and Je = the terms of J that e owns (its
// pairs with j > e and its e-n terms), so that sum_e Je = J.  Pade form
// U = a r / (1 + b r): U' = a / (1 + b r)^2, U'' = -2 a b / (1 + b r)^3,
// lap U(|r_e - x|) = U'' + 2 U' / r, grad U = U' (r_e - x) / r.
__device__ __forceinline__ void jastrow_e(const SysDev &s, const double *__restrict__ Rw, int e, int lane,
                                          double &g0, double &g1, double &g2, double &L, double &Je)
{
    const double rx = Rw[3 * e], ry = Rw[3 * e + 1], rz = Rw[3 * e + 2];
    const bool up = e < s.n_up;
    g0 = g1 = g2 = L = Je = 0.0;
    auto term = [&](double dx, double dy, double dz, double a, double b, bool own) {
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        const double q = 1.0 + b * r, iq = 1.0 / q;
        const double u1 = a * iq * iq, u2 = -2.0 * a * b * iq * iq * iq;
        const double f = u1 / r;
        g0 += f * dx; g1 += f * dy; g2 += f * dz;
        L += u2 + 2.0 * f;
        if (own) Je += a * r * iq;
    };
    for (int j = lane; j < s.n_elec; j += 32) {
        if (j == e) continue;
        const double a = ((j < s.n_up) == up) ? s.ja_par : s.ja_anti;
        term(rx - Rw[3 * j], ry - Rw[3 * j + 1], rz - Rw[3 * j + 2], a, s.jb_ee, j > e);
    }
    for (int at = lane; at < s.n_atom; at += 32)
        term(rx - s.Q[3 * at], ry - s.Q[3 * at + 1], rz - s.Q[3 * at + 2], -s.ja_en[at], s.jb_en[at], true);
    g0 = warp_sum(g0); g1 = warp_sum(g1); g2 = warp_sum(g2);
    L = warp_sum(L);
    Je = warp_sum(Je);
}

template <typename TG>
__global__ void __launch_bounds__(kEnThreads) k_drift_energy(SysDev s, const double *__restrict__ R,
                                                             const double *__restrict__ Dinv,
                                                             const TG *__restrict__ Cg, CView cv,
                                                             const double *__restrict__ logabs2,
                                                             const double *__restrict__ sign2,
                                                             const uint32_t *__restrict__ sing,
                                                             qmc_eval_out o, int w_off, const float2 *__restrict__ Q2)
{
    constexpr bool kMixed = std::is_same<TG, float>::value;
    extern __shared__ __align__(16) unsigned char en_smem[];   // mixed: positions, nuclei, charges
    __shared__ double red[4][kEnWarps];
    __shared__ int s_nonfinite;
    const int w = blockIdx.x;
    const int wg = w + w_off;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int N = s.n_elec;
    const size_t msz = (size_t)s.n_up * s.n_up + (size_t)s.n_dn * s.n_dn;
    const double *Rw = R + (size_t)w * N * 3;

    double lap_acc = 0.0, jas_acc = 0.0;
    for (int e = wid; e < N; e += kEnWarps) {
        double b0 = 0.0, b1 = 0.0, b2 = 0.0, b3 = 0.0;
        if (cv.vd) {             // C-free variant: drift and Laplacian of the determinants already formed
            const double *v = cv.vd + ((size_t)w * N + e) * 4;
            b0 = v[0]; b1 = v[1]; b2 = v[2]; b3 = v[3];
        } else {
            dets_drift_lap<kMixed>(s, Dinv, Cg, cv, w, e, lane, msz, b0, b1, b2, b3);
        }
        double g0 = 0.0, g1 = 0.0, g2 = 0.0, L = 0.0, Je = 0.0;
        if (s.jas) jastrow_e(s, Rw, e, lane, g0, g1, g2, L, Je);
        if (lane == 0) {
            double *dr = o.drift + ((size_t)wg * N + e) * 3;
            dr[0] = b0 + g0; dr[1] = b1 + g1; dr[2] = b2 + g2;
            // lap_e Psi / Psi with Psi = e^J Det: lap J + |grad J|^2 + 2 grad J . grad Det / Det + lap Det / Det
            lap_acc += b3 + L + (g0 * g0 + g1 * g1 + g2 * g2) + 2.0 * (g0 * b0 + g1 * b1 + g2 * b2);
            jas_acc += Je;
        }
    }
    double ven = 0.0, vee = 0.0;
    if constexpr (kMixed) {
        float2 *rs = reinterpret_cast<float2 *>(en_smem);
        float2 *qs = rs + 3 * N;
        float *zs = reinterpret_cast<float *>(qs + 3 * s.n_atom);
        if (t == 0) s_nonfinite = 0;
        __syncthreads();
        int bad = 0;
        for (int q = t; q < 3 * N; q += kEnThreads) {
            const double x = Rw[q];
            bad |= !isfinite(x);
            rs[q] = ff::from_double(x);
        }
        for (int q = t; q < 3 * s.n_atom; q += kEnThreads) qs[q] = Q2[q];
        for (int a = t; a < s.n_atom; a += kEnThreads) zs[a] = (float)s.Z[a];
        if (bad) s_nonfinite = 1;
        __syncthreads();
        coulomb_ff(s, rs, qs, zs, ven, vee);
    } else {
        for (int e = wid; e < N; e += kEnWarps) {
            const double rx = Rw[3 * e], ry = Rw[3 * e + 1], rz = Rw[3 * e + 2];
            for (int a = lane; a < s.n_atom; a += 32) {
                const double dx = rx - s.Q[3 * a], dy = ry - s.Q[3 * a + 1], dz = rz - s.Q[3 * a + 2];
                ven -= s.Z[a] * rsqrt(dx * dx + dy * dy + dz * dz);
            }
            for (int j = e + 1 + lane; j < N; j += 32) {
                const double dx = rx - Rw[3 * j], dy = ry - Rw[3 * j + 1], dz = rz - Rw[3 * j + 2];
                vee += rsqrt(dx * dx + dy * dy + dz * dz);
            }
        }
    }
    ven = warp_sum(ven);
    vee = warp_sum(vee);
    if (lane == 0) { red[0][wid] = lap_acc; red[1][wid] = ven; red[2][wid] = vee; red[3][wid] = jas_acc; }
    __syncthreads();
    if (t == 0) {
        double lap = 0.0, Ven = 0.0, Vee = 0.0, Jt = 0.0;
        for (int q = 0; q < kEnWarps; ++q) { lap += red[0][q]; Ven += red[1][q]; Vee += red[2][q]; Jt += red[3][q]; }
        const double T = -0.5 * lap;
        const double el = T + Ven + Vee + s.vnn;
        // a spin with no electrons contributes det = 1
        const double la0 = s.n_up ? logabs2[2 * w] : 0.0, la1 = s.n_dn ? logabs2[2 * w + 1] : 0.0;
        const double sg0 = s.n_up ? sign2[2 * w] : 1.0, sg1 = s.n_dn ? sign2[2 * w + 1] : 1.0;
        uint32_t st = sing[w];
        const bool singular = (st & (QMC_STATUS_SINGULAR_UP | QMC_STATUS_SINGULAR_DN)) != 0;
        bool finite_in = true;
        if constexpr (kMixed) finite_in = !s_nonfinite;
        else
            for (int q = 0; q < 3 * N; ++q) finite_in = finite_in && isfinite(Rw[q]);
        if (!finite_in) st |= QMC_STATUS_NONFINITE;
        if (!singular && !(isfinite(el) && isfinite(la0) && isfinite(la1) && isfinite(Jt))) st |= QMC_STATUS_NONFINITE;
        o.logpsi[wg] = singular ? -INFINITY : la0 + la1 + Jt;     // log|Psi| = log|Det_up| + log|Det_dn| + J
        o.sign[wg] = singular ? 0.0 : sg0 * sg1;
        if (o.logabs) { o.logabs[2 * wg] = la0; o.logabs[2 * wg + 1] = la1; }
        o.e_loc[wg] = el;
        if (o.e_parts) {
            o.e_parts[4 * wg] = T; o.e_parts[4 * wg + 1] = Ven;
            o.e_parts[4 * wg + 2] = Vee; o.e_parts[4 * wg + 3] = s.vnn;
        }
        o.status[wg] = st;
    }
}

cudaError_t launch_drift_energy(const SysDev &s, int nw, const double *R, const double *Dinv, const CView &cv,
                                const double *logabs2, const double *sign2, const uint32_t *sing,
                                const qmc_eval_out &o, int w_off, cudaStream_t st, const float2 *Q2)
{
    if (nw == 0) return cudaSuccess;
    if (cv.g_f32) {
        const size_t sm = sizeof(float2) * 3 * ((size_t)s.n_elec + s.n_atom) + sizeof(float) * (size_t)s.n_atom;
        cudaError_t e = cudaFuncSetAttribute(k_drift_energy<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sm);
        if (e != cudaSuccess) return e;
        k_drift_energy<float><<<nw, kEnThreads, sm, st>>>(s, R, Dinv, static_cast<const float *>(cv.g), cv,
                                                          logabs2, sign2, sing, o, w_off, Q2);
    } else {
        k_drift_energy<double><<<nw, kEnThreads, 0, st>>>(s, R, Dinv, static_cast<const double *>(cv.g), cv,
                                                           logabs2, sign2, sing, o, w_off, nullptr);
    }
    return cudaGetLastError();
}

}  // namespace qmc
