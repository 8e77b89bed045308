// Steps a1-a3 of the plain FP64 path.
//
// k_screen_ao: screening + AO values/gradients/Laplacians written out (for
//   inspection and parity tests).
// k_contract_f64: fused screening + AO evaluation + the five products
//   C_l[e][k] = sum_{mu in list(e)} B_l[mu] A[mu][k]  (Sec. III, Eq. "abc";
//   the paper's sparse-B x dense-A loop: electron, non-zero AO, MO).  One CTA
//   per (walker, electron); the AO values live in shared memory only, so B
//   never reaches HBM.  Each thread owns MOs k = t + 128 j and keeps the five
//   accumulators of each in registers; one A element feeds five DFMAs.
#include "qmc_device.cuh"

namespace qmc {

constexpr int kAoThreads = 128;
constexpr int kAoChunk = 512;   // AO values staged per pass (5 x 512 doubles = 20 KB)

__global__ void __launch_bounds__(kAoThreads) k_screen_ao(SysDev s, const double *__restrict__ R,
                                                          int cap, int32_t *cnt, int32_t *idx,
                                                          double *B)
{
    extern __shared__ int idx_s[];   // [n_ao]
    __shared__ int warp_s[kAoThreads / 32];
    const int e = blockIdx.x, w = blockIdx.y;
    const double *r = R + ((size_t)w * s.n_elec + e) * 3;
    const double rx = r[0], ry = r[1], rz = r[2];
    const int K = screen_electron<kAoThreads>(s, rx, ry, rz, idx_s, s.n_ao, warp_s);
    const size_t row = (size_t)w * s.n_elec + e;
    if (threadIdx.x == 0) cnt[row] = K;
    const int Kw = min(K, cap);
    for (int k = threadIdx.x; k < Kw; k += kAoThreads) {
        const int mu = idx_s[k];
        idx[row * cap + k] = mu;
        if (B) {
            double v[5];
            ao_eval_f64(s, mu, rx, ry, rz, v);
#pragma unroll
            for (int l = 0; l < 5; ++l) B[(row * 5 + l) * cap + k] = v[l];
        }
    }
}

template <int NJ>
__global__ void __launch_bounds__(kAoThreads) k_contract_f64(SysDev s, const double *__restrict__ R,
                                                             double *__restrict__ X,
                                                             double *__restrict__ Cd)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *B_s = reinterpret_cast<double *>(smem_raw);             // [5][kAoChunk]
    int *idx_s = reinterpret_cast<int *>(B_s + 5 * kAoChunk);       // [n_ao]
    __shared__ int warp_s[kAoThreads / 32];

    const int e = blockIdx.x, w = blockIdx.y;
    const int spin = e >= s.n_up;
    const int ei = spin ? e - s.n_up : e;
    const int ns = spin ? s.n_dn : s.n_up;
    const double *__restrict__ A = s.A64[spin];
    const double *r = R + ((size_t)w * s.n_elec + e) * 3;
    const double rx = r[0], ry = r[1], rz = r[2];

    const int K = screen_electron<kAoThreads>(s, rx, ry, rz, idx_s, s.n_ao, warp_s);

    double acc[5][NJ];
#pragma unroll
    for (int l = 0; l < 5; ++l)
#pragma unroll
        for (int j = 0; j < NJ; ++j) acc[l][j] = 0.0;

    const int t = threadIdx.x;
    for (int k0 = 0; k0 < K; k0 += kAoChunk) {
        const int kc = min(kAoChunk, K - k0);
        for (int m = t; m < kc; m += kAoThreads) {
            double v[5];
            ao_eval_f64(s, idx_s[k0 + m], rx, ry, rz, v);
#pragma unroll
            for (int l = 0; l < 5; ++l) B_s[l * kAoChunk + m] = v[l];
        }
        __syncthreads();
        // MO slots j whose whole warp lies beyond ns are skipped (warp-uniform)
        const int kwarp = t & ~31;
#pragma unroll 2
        for (int m = 0; m < kc; ++m) {
            const double *__restrict__ arow = A + (size_t)idx_s[k0 + m] * ns;
            double a[NJ];
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                const int k = t + kAoThreads * j;
                a[j] = (k < ns) ? __ldg(arow + k) : 0.0;
            }
            double b[5];
#pragma unroll
            for (int l = 0; l < 5; ++l) b[l] = B_s[l * kAoChunk + m];
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                if (kwarp + kAoThreads * j < ns) {
#pragma unroll
                    for (int l = 0; l < 5; ++l) acc[l][j] = fma(a[j], b[l], acc[l][j]);
                }
            }
        }
        __syncthreads();
    }

    // X: [w][n_up^2 + n_dn^2] (C1, row e), Cd: [w][4][...] (C2..C5)
    const size_t msz = (size_t)s.n_up * s.n_up + (size_t)s.n_dn * s.n_dn;
    const size_t soff = spin ? (size_t)s.n_up * s.n_up : 0;
    const size_t nss = (size_t)ns * ns;
    double *xrow = X + (size_t)w * msz + soff + (size_t)ei * ns;
    double *crow = Cd + (size_t)w * 4 * msz + 4 * soff + (size_t)ei * ns;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int k = t + kAoThreads * j;
        if (k < ns) {
            xrow[k] = acc[0][j];
#pragma unroll
            for (int l = 1; l < 5; ++l) crow[(l - 1) * nss + k] = acc[l][j];
        }
    }
}

cudaError_t launch_screen_ao(const SysDev &s, int nw, const double *R, int cap, int32_t *cnt,
                             int32_t *idx, double *B, cudaStream_t st)
{
    if (nw == 0 || s.n_elec == 0) return cudaSuccess;
    const size_t sm = sizeof(int) * (size_t)s.n_ao;
    dim3 grid(s.n_elec, nw);
    k_screen_ao<<<grid, kAoThreads, sm, st>>>(s, R, cap, cnt, idx, B);
    return cudaGetLastError();
}

template <int NJ>
static cudaError_t launch_contract_nj(const SysDev &s, int nw, const double *R, double *X, double *Cd,
                                      cudaStream_t st)
{
    const size_t sm = sizeof(double) * 5 * kAoChunk + sizeof(int) * (size_t)s.n_ao;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_contract_f64<NJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             64 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grid(s.n_elec, nw);
    k_contract_f64<NJ><<<grid, kAoThreads, sm, st>>>(s, R, X, Cd);
    return cudaGetLastError();
}

cudaError_t launch_contract_f64(const SysDev &s, int nw, const double *R, double *X, double *Cd,
                                cudaStream_t st)
{
    if (nw == 0 || s.n_elec == 0) return cudaSuccess;
    const int nmax = s.n_up > s.n_dn ? s.n_up : s.n_dn;
    const int nj = (nmax + kAoThreads - 1) / kAoThreads;
    switch (nj) {
    case 1: return launch_contract_nj<1>(s, nw, R, X, Cd, st);
    case 2: return launch_contract_nj<2>(s, nw, R, X, Cd, st);
    case 3: return launch_contract_nj<3>(s, nw, R, X, Cd, st);
    case 4: return launch_contract_nj<4>(s, nw, R, X, Cd, st);
    case 5: return launch_contract_nj<5>(s, nw, R, X, Cd, st);
    case 6: return launch_contract_nj<6>(s, nw, R, X, Cd, st);
    case 7: return launch_contract_nj<7>(s, nw, R, X, Cd, st);
    case 8: return launch_contract_nj<8>(s, nw, R, X, Cd, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace qmc
