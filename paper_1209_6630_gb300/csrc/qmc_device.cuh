// Device helpers shared by the kernels: screening (Sec. III) and Cartesian
// Gaussian AO evaluation (Sec. II.C, AO form).
#pragma once

#include "qmc_internal.cuh"

namespace qmc {

__device__ __forceinline__ int ncart(int L) { return (L + 1) * (L + 2) / 2; }

// Squared distance rounded exactly as ((dx*dx) + (dy*dy)) + (dz*dz), each
// operation correctly rounded and never fused: the screening decision
// d2 < R2 must not depend on FMA contraction.
__device__ __forceinline__ double sqdist_rn(double rx, double ry, double rz, const double *q)
{
    double dx = __dsub_rn(rx, q[0]);
    double dy = __dsub_rn(ry, q[1]);
    double dz = __dsub_rn(rz, q[2]);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Exclusive prefix sum over the block of `v`; *total receives the sum.
template <int NT>
__device__ __forceinline__ int block_excl_scan(int v, int *warp_s, int *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_s[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int s = (lane < NT / 32) ? warp_s[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < NT / 32) warp_s[lane] = s;   // inclusive warp totals
    }
    __syncthreads();
    int base = (wid > 0) ? warp_s[wid - 1] : 0;
    *total = warp_s[NT / 32 - 1];
    __syncthreads();
    return base + x - v;
}

// Ascending list of the AOs whose shell is active for an electron at r
// (Sec. III): shell s of atom a is active iff d2 < R2_s; the atom is skipped
// when d2 >= R2_atom (the paper's atomic radius, identical decisions).
// Thread t scans a contiguous run of at most 64 shells, so the compaction
// keeps the global order.  Returns the list length K (all threads).
template <int NT>
__device__ int screen_electron(const SysDev &s, double rx, double ry, double rz, int *idx_s,
                               int cap_s, int *warp_s)
{
    const int t = threadIdx.x;
    const int per = (s.n_shell + NT - 1) / NT;   // <= 64, checked at load
    const int sh0 = min(t * per, s.n_shell), sh1 = min(sh0 + per, s.n_shell);
    unsigned long long mask = 0ull;
    int nao = 0, last_a = -1;
    bool atom_in = false;
    double d2 = 0.0;
    for (int sh = sh0; sh < sh1; ++sh) {
        const int a = s.sh_atom[sh];
        if (a != last_a) {
            last_a = a;
            d2 = sqdist_rn(rx, ry, rz, s.Q + 3 * a);
            atom_in = d2 < s.atom_R2[a];
        }
        if (atom_in && d2 < s.sh_R2[sh]) {
            mask |= 1ull << (sh - sh0);
            nao += ncart(s.sh_L[sh]);
        }
    }
    int total;
    int off = block_excl_scan<NT>(nao, warp_s, &total);
    while (mask) {
        const int b = __ffsll((long long)mask) - 1;
        mask &= mask - 1;
        const int sh = sh0 + b;
        const int a0 = s.sh_ao0[sh], nc = ncart(s.sh_L[sh]);
        for (int c = 0; c < nc; ++c, ++off)
            if (off < cap_s) idx_s[off] = a0 + c;
    }
    __syncthreads();
    return total;
}

__device__ __forceinline__ double ipow_small(double x, int n)
{
    switch (n) {
    case 0: return 1.0;
    case 1: return x;
    case 2: return x * x;
    case 3: return x * x * x;
    case 4: { double y = x * x; return y * y; }
    default: return 0.0;   // n < 0: the derivative term vanishes
    }
}

// Value, gradient and Laplacian of AO mu at r, FP64.
//   chi = c P(d) g(d2),  P = dx^nx dy^ny dz^nz,  g = sum_p c_p e^{-gamma_p d2}
//   d_l chi = c (d_l P g - 2 d_l P gd),            gd = sum_p c_p gamma_p e_p
//   lap chi = c (lap P g + P (gl - 4 L gd)),        gl = sum_p c_p (4 gamma_p^2 d2 - 6 gamma_p) e_p
// (the cross term 2 grad P . grad g = -4 gd (d . grad P) = -4 L gd P by
// Euler's theorem for the degree-L monomial P).
__device__ __forceinline__ void ao_eval_f64(const SysDev &s, int mu, double rx, double ry, double rz,
                                            double out[5])
{
    const int sh = s.ao_shell[mu];
    const int a = s.sh_atom[sh];
    const double dx = rx - s.Q[3 * a], dy = ry - s.Q[3 * a + 1], dz = rz - s.Q[3 * a + 2];
    const double d2 = dx * dx + dy * dy + dz * dz;
    double g = 0.0, gd = 0.0, gl = 0.0;
    const int p0 = s.sh_pstart[sh], np = s.sh_nprim[sh];
    for (int p = 0; p < np; ++p) {
        const double gam = s.pg[p0 + p];
        const double ce = s.pc[p0 + p] * exp(-gam * d2);
        g += ce;
        gd += gam * ce;
        gl += (4.0 * gam * d2 - 6.0) * gam * ce;
    }
    const int pw = s.ao_pow[mu];
    const int nx = pw & 255, ny = (pw >> 8) & 255, nz = (pw >> 16) & 255;
    const int L = nx + ny + nz;
    const double px = ipow_small(dx, nx), py = ipow_small(dy, ny), pz = ipow_small(dz, nz);
    const double P = px * py * pz;
    const double dpx = nx ? nx * ipow_small(dx, nx - 1) : 0.0;
    const double dpy = ny ? ny * ipow_small(dy, ny - 1) : 0.0;
    const double dpz = nz ? nz * ipow_small(dz, nz - 1) : 0.0;
    const double ddx = nx > 1 ? nx * (nx - 1) * ipow_small(dx, nx - 2) : 0.0;
    const double ddy = ny > 1 ? ny * (ny - 1) * ipow_small(dy, ny - 2) : 0.0;
    const double ddz = nz > 1 ? nz * (nz - 1) * ipow_small(dz, nz - 2) : 0.0;
    const double c = s.ao_scale[mu];
    const double m2gd = -2.0 * gd;
    out[0] = c * P * g;
    out[1] = c * (dpx * py * pz * g + m2gd * dx * P);
    out[2] = c * (px * dpy * pz * g + m2gd * dy * P);
    out[3] = c * (px * py * dpz * g + m2gd * dz * P);
    const double lapP = ddx * py * pz + px * ddy * pz + px * py * ddz;
    out[4] = c * (lapP * g + P * (gl - 4.0 * L * gd));
}

// Value of AO mu at r, FP64.
__device__ __forceinline__ double ao_value_f64(const SysDev &s, int mu, double rx, double ry, double rz)
{
    const int sh = s.ao_shell[mu];
    const int a = s.sh_atom[sh];
    const double dx = rx - s.Q[3 * a], dy = ry - s.Q[3 * a + 1], dz = rz - s.Q[3 * a + 2];
    const double d2 = dx * dx + dy * dy + dz * dz;
    double g = 0.0;
    const int p0 = s.sh_pstart[sh], np = s.sh_nprim[sh];
    for (int p = 0; p < np; ++p) g += s.pc[p0 + p] * exp(-s.pg[p0 + p] * d2);
    const int pw = s.ao_pow[mu];
    return s.ao_scale[mu] * ipow_small(dx, pw & 255) * ipow_small(dy, (pw >> 8) & 255) *
           ipow_small(dz, (pw >> 16) & 255) * g;
}

}  // namespace qmc
