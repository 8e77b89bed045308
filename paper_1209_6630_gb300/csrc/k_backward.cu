// Step a7: adjoint of log|Psi| with respect to the MO coefficients, FP64.
//
//   dA_s[mu][k] = sum_w g_w sum_{e in s} chi_mu(r_{w,e}) (D^-1)_{w,ek}
//
// (d log|det D| / d D_{ke} = (D^-1)_{ek} and D_{ke} = sum_mu a_{k mu} chi_mu(r_e),
// the cofactor identity behind the drift formula of Sec. II.C.)  chi is
// recomputed from R with the forward pass's exact screening decisions; the
// AO values are never stored.
//
// One CTA per (atom a, block of 128 MOs, spin).  The CTA owns the rows of dA
// belonging to the atom's AOs, so no atomics are needed: it scans every
// (walker, electron) pair, keeps those inside the atomic radius (same
// correctly rounded d2 as the forward screening), evaluates the atom's active
// AOs for a batch of hits in shared memory and accumulates
// acc[mu] += g_w chi_mu (D^-1)_{ek} in registers (thread = MO k).
#include "qmc_device.cuh"

namespace qmc {

constexpr int kBwThreads = 128;
constexpr int kBwBatch = 128;   // hits buffered before an accumulation pass

template <int MAXAO>
__global__ void __launch_bounds__(kBwThreads) k_backward_f64(SysDev s, int nw, const double *__restrict__ R,
                                                             const double *__restrict__ dinv,
                                                             const double *__restrict__ gw,
                                                             double *__restrict__ dA_up,
                                                             double *__restrict__ dA_dn)
{
    __shared__ int hit_w[kBwBatch + kBwThreads], hit_e[kBwBatch + kBwThreads];
    extern __shared__ double chi_s[];   // [kBwBatch + kBwThreads][MAXAO]
    __shared__ int warp_s[kBwThreads / 32];
    __shared__ int s_nhit;

    const int a = blockIdx.x, spin = blockIdx.z;
    const int ns = spin ? s.n_dn : s.n_up;
    const int e0 = spin ? s.n_up : 0;
    const int k = blockIdx.y * kBwThreads + threadIdx.x;
    if (blockIdx.y * kBwThreads >= ns) return;
    const int t = threadIdx.x;
    const int sh0 = s.atom_sh0[a], sh1 = s.atom_sh0[a + 1];
    if (sh1 == sh0) return;   // an atom without basis functions owns no rows of dA
    const int ao0 = s.sh_ao0[sh0];
    const int nao = s.sh_ao0[sh1 - 1] + ncart(s.sh_L[sh1 - 1]) - ao0;
    const double ra2 = s.atom_R2[a];
    const double *q = s.Q + 3 * a;
    const size_t msz = (size_t)s.n_up * s.n_up + (size_t)s.n_dn * s.n_dn;
    const size_t soff = spin ? (size_t)s.n_up * s.n_up : 0;

    double acc[MAXAO];
#pragma unroll
    for (int m = 0; m < MAXAO; ++m) acc[m] = 0.0;
    if (t == 0) s_nhit = 0;
    __syncthreads();

    const long long npair = (long long)nw * ns;
    for (long long q0 = 0; q0 < npair; q0 += kBwThreads) {
        const long long qq = q0 + t;
        int w = 0, ei = 0, hit = 0;
        if (qq < npair) {
            w = (int)(qq / ns);
            ei = (int)(qq - (long long)w * ns);
            if (gw[w] != 0.0) {
                const double *r = R + ((size_t)w * s.n_elec + e0 + ei) * 3;
                hit = sqdist_rn(r[0], r[1], r[2], q) < ra2;
            }
        }
        int total;
        const int base = s_nhit;
        const int off = block_excl_scan<kBwThreads>(hit, warp_s, &total);
        if (hit) { hit_w[base + off] = w; hit_e[base + off] = ei; }
        __syncthreads();
        const int nh = base + total;
        const bool last = q0 + kBwThreads >= npair;
        if (nh >= kBwBatch || (last && nh > 0)) {
            // AO values (times g_w) of the atom's active shells for every hit
            for (int p = t; p < nh * MAXAO; p += kBwThreads) {
                const int h = p / MAXAO, m = p - h * MAXAO;
                double v = 0.0;
                if (m < nao) {
                    const int mu = ao0 + m;
                    const double *r = R + ((size_t)hit_w[h] * s.n_elec + e0 + hit_e[h]) * 3;
                    const double d2 = sqdist_rn(r[0], r[1], r[2], q);
                    if (d2 < s.sh_R2[s.ao_shell[mu]])
                        v = gw[hit_w[h]] * ao_value_f64(s, mu, r[0], r[1], r[2]);
                }
                chi_s[p] = v;
            }
            __syncthreads();
            if (k < ns) {
                for (int h = 0; h < nh; ++h) {
                    const double dv = dinv[(size_t)hit_w[h] * msz + soff + (size_t)hit_e[h] * ns + k];
                    const double *c = chi_s + h * MAXAO;
#pragma unroll
                    for (int m = 0; m < MAXAO; ++m) acc[m] = fma(c[m], dv, acc[m]);
                }
            }
            __syncthreads();
            if (t == 0) s_nhit = 0;
        } else if (t == 0) {
            s_nhit = nh;
        }
        __syncthreads();
    }
    if (k < ns) {
        double *dA = spin ? dA_dn : dA_up;
#pragma unroll
        for (int m = 0; m < MAXAO; ++m)
            if (m < nao) dA[(size_t)(ao0 + m) * ns + k] = acc[m];
    }
}

template <int MAXAO>
static cudaError_t launch_bw(const SysDev &s, int nw, const double *R, const double *dinv, const double *g,
                             double *dA_up, double *dA_dn, cudaStream_t st)
{
    const int nmax = s.n_up > s.n_dn ? s.n_up : s.n_dn;
    dim3 grid(s.n_atom, (nmax + kBwThreads - 1) / kBwThreads, 2);
    const size_t sm = sizeof(double) * (size_t)(kBwBatch + kBwThreads) * MAXAO;
    cudaError_t e = cudaFuncSetAttribute(k_backward_f64<MAXAO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    k_backward_f64<MAXAO><<<grid, kBwThreads, sm, st>>>(s, nw, R, dinv, g, dA_up, dA_dn);
    return cudaGetLastError();
}

cudaError_t launch_backward_f64(const SysDev &s, int nw, const double *R, const double *dinv,
                                const double *g, double *dA_up, double *dA_dn, cudaStream_t st,
                                int max_ao_per_atom)
{
    if (max_ao_per_atom <= 16) return launch_bw<16>(s, nw, R, dinv, g, dA_up, dA_dn, st);
    if (max_ao_per_atom <= 32) return launch_bw<32>(s, nw, R, dinv, g, dA_up, dA_dn, st);
    return cudaErrorInvalidValue;
}

}  // namespace qmc
