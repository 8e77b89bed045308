// The Monte Carlo step around the walker evaluation (Sec. II.A, II.B):
//   Eq. (1)  drift-diffusion move R' = R + tau b(R) + sqrt(tau) eta
//   Eq. (3)  branching weight w = exp(-tau/2 [(E_L(R') - E_T) + (E_L(R) - E_T)])
//            with the fixed-node rule (a move across a node of Psi_T is not made)
//   Sec. II.B constant-population reconfiguration: M walkers drawn among the M
//            walkers with probabilities w_k / sum_i w_i
//
// Random numbers: Philox4x64-10 (Salmon et al., SC'11), counter-based, so
// every (walker, component, step) has its own numbers whatever the launch
// shape.  Streams: move key (seed, 0), counter (block j, walker, step, 0), four
// normals per block by two Box-Muller pairs; draws key (seed, 1), counter
// (j >> 2, step, 0, 0), output j & 3 is draw j's 64-bit uniform integer.
//
// The drawing is exact integer arithmetic: q_k = floor(2^40 w_k / w_max),
// C_k = q_0 + ... + q_k in 64-bit integers (a block scan, exact in any
// order), t_j = high word of U_j * C_{M-1}, draw j = first k with C_k > t_j.
// The drawn indices are therefore a function of the weights only.
//
// Kernels: k_dmc_move (one thread per four components of a walker: HBM-bound,
// 72 N bytes per walker), k_dmc_weight (one thread per walker),
// k_srmc (one CTA: max, block scan, binary searches), k_dmc_gather (one CTA
// per new walker: copies the drawn walker's state, 96 N + 36 bytes).
#include "qmc_internal.cuh"

namespace qmc {

namespace {

// One Philox4x64-10 block: ten rounds, key bumped by the Weyl constants.
__device__ __forceinline__ void philox4x64(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0,
                                           uint64_t k1, uint64_t out[4])
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t lo0 = 0xD2E7470EE14C6C93ull * c0, hi0 = __umul64hi(0xD2E7470EE14C6C93ull, c0);
        const uint64_t lo1 = 0xCA5A826395121157ull * c2, hi1 = __umul64hi(0xCA5A826395121157ull, c2);
        const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B97F4A7C15ull;
        k1 += 0xBB67AE8584CAA73Bull;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Box-Muller on two 64-bit uniform integers: u1 in (0, 1], u2 in [0, 1).
__device__ __forceinline__ void box_muller(uint64_t x0, uint64_t x1, double &n0, double &n1)
{
    const double u1 = (double)((x0 >> 11) + 1) * 0x1p-53;
    const double u2 = (double)(x1 >> 11) * 0x1p-53;
    const double r = sqrt(__dmul_rn(-2.0, log(u1)));
    const double th = __dmul_rn(6.283185307179586476925286766559, u2);
    double s, c;
    sincos(th, &s, &c);
    n0 = __dmul_rn(r, c);
    n1 = __dmul_rn(r, s);
}

__device__ __forceinline__ uint64_t step_of(uint64_t step, const uint64_t *step_ptr)
{
    return step_ptr ? *step_ptr : step;
}

__global__ void k_dmc_move(int nw, int nc, const double *__restrict__ R, const double *__restrict__ drift,
                           double tau, double sqrt_tau, uint64_t seed, uint64_t step, const uint64_t *step_ptr,
                           double *__restrict__ Rn)
{
    const int nb = (nc + 3) >> 2;
    const size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (q >= (size_t)nw * nb) return;
    const int w = (int)(q / nb), j = (int)(q - (size_t)w * nb);
    uint64_t x[4];
    philox4x64((uint64_t)j, (uint64_t)w, step_of(step, step_ptr), 0, seed, 0, x);
    double eta[4];
    box_muller(x[0], x[1], eta[0], eta[1]);
    box_muller(x[2], x[3], eta[2], eta[3]);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int c = 4 * j + i;
        if (c >= nc) break;
        const size_t o = (size_t)w * nc + c;
        // ((R + tau b) + sqrt(tau) eta), rounded as written (no fused multiply-add)
        Rn[o] = __dadd_rn(__dadd_rn(R[o], __dmul_rn(tau, drift[o])), __dmul_rn(sqrt_tau, eta[i]));
    }
}

__global__ void k_dmc_weight(int nw, const double *__restrict__ e_old, const double *__restrict__ s_old,
                             const uint32_t *__restrict__ st_old, const double *__restrict__ e_new,
                             const double *__restrict__ s_new, const uint32_t *__restrict__ st_new,
                             double half_tau, double e_trial, const double *e_trial_ptr, double *__restrict__ weight,
                             uint32_t *__restrict__ accept)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nw) return;
    const double eT = e_trial_ptr ? *e_trial_ptr : e_trial;
    const bool valid_old = st_old[w] == 0u && s_old[w] != 0.0;
    const bool acc = valid_old && st_new[w] == 0u && s_new[w] == s_old[w];
    accept[w] = acc ? 1u : 0u;
    if (!valid_old) {
        weight[w] = 0.0;
        return;
    }
    const double en = acc ? e_new[w] : e_old[w];
    const double s = __dadd_rn(__dsub_rn(en, eT), __dsub_rn(e_old[w], eT));
    weight[w] = exp(-__dmul_rn(s, half_tau));
}

constexpr int kSrThreads = 1024;

__device__ __forceinline__ bool live(double x) { return isfinite(x) && x > 0.0; }

// One CTA.  stats (optional, device [4]): sum of the counted weights, their
// number, sum of w_k E_L of the kept state (e_sel: accept ? e_new : e_old), the
// number of accepted moves.
__global__ void __launch_bounds__(kSrThreads) k_srmc(int nw, const double *__restrict__ weight, uint64_t seed,
                                                     uint64_t step, const uint64_t *step_ptr,
                                                     unsigned long long *__restrict__ C, int *__restrict__ idx,
                                                     double *__restrict__ stats, const double *__restrict__ e_new,
                                                     const double *__restrict__ e_old,
                                                     const uint32_t *__restrict__ accept)
{
    __shared__ double s_max[32], s_sum[32], s_swe[32];
    __shared__ int s_alive[32], s_acc[32];
    __shared__ unsigned long long s_scan[kSrThreads];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int per = (nw + kSrThreads - 1) / kSrThreads;
    const int k0 = min(nw, t * per), k1 = min(nw, k0 + per);
    double m = 0.0, sum = 0.0, swe = 0.0;
    int alive = 0, nacc = 0;
    for (int k = k0; k < k1; ++k) {
        const double x = weight[k];
        if (live(x)) {
            m = fmax(m, x);
            sum += x;
            ++alive;
            if (e_new) swe += x * (accept[k] ? e_new[k] : e_old[k]);
        }
        if (accept) nacc += accept[k] ? 1 : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        swe += __shfl_xor_sync(0xffffffffu, swe, o);
        alive += __shfl_xor_sync(0xffffffffu, alive, o);
        nacc += __shfl_xor_sync(0xffffffffu, nacc, o);
    }
    if (lane == 0) { s_max[wid] = m; s_sum[wid] = sum; s_swe[wid] = swe; s_alive[wid] = alive; s_acc[wid] = nacc; }
    __syncthreads();
    if (wid == 0) {
        m = s_max[lane]; sum = s_sum[lane]; swe = s_swe[lane]; alive = s_alive[lane]; nacc = s_acc[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
            sum += __shfl_xor_sync(0xffffffffu, sum, o);
            swe += __shfl_xor_sync(0xffffffffu, swe, o);
            alive += __shfl_xor_sync(0xffffffffu, alive, o);
            nacc += __shfl_xor_sync(0xffffffffu, nacc, o);
        }
        if (lane == 0) {
            s_max[0] = m;
            if (stats) {
                stats[0] = sum;
                stats[1] = (double)alive;
                stats[2] = swe;
                stats[3] = (double)nacc;
            }
        }
    }
    __syncthreads();
    const double wmax = s_max[0];
    const uint64_t st = step_of(step, step_ptr);
    if (!(wmax > 0.0)) {                          // every weight 0: keep the population
        for (int j = t; j < nw; j += kSrThreads) idx[j] = j;
        return;
    }
    // q_k = floor(2^40 w_k / w_max): one rounded division, then an exact scaling
    unsigned long long run = 0;
    for (int k = k0; k < k1; ++k) {
        const double x = weight[k];
        const unsigned long long q = live(x) ? (unsigned long long)(__ddiv_rn(x, wmax) * 0x1p40) : 0ull;
        run += q;
        C[k] = run;                               // local inclusive sums, offset below
    }
    s_scan[t] = run;
    __syncthreads();
    for (int o = 1; o < kSrThreads; o <<= 1) {    // inclusive scan of the per-thread totals (exact)
        const unsigned long long v = t >= o ? s_scan[t - o] : 0ull;
        __syncthreads();
        s_scan[t] += v;
        __syncthreads();
    }
    const unsigned long long off = t > 0 ? s_scan[t - 1] : 0ull;
    for (int k = k0; k < k1; ++k) C[k] += off;
    const unsigned long long T = s_scan[kSrThreads - 1];
    __syncthreads();                              // C complete (global writes of this CTA, visible after the barrier)
    __threadfence_block();
    for (int j = t; j < nw; j += kSrThreads) {
        uint64_t x[4];
        philox4x64((uint64_t)(j >> 2), st, 0, 0, seed, 1, x);
        const unsigned long long tj = __umul64hi(x[j & 3], T);
        int lo = 0, hi = nw - 1;                  // first k with C_k > tj (C_{nw-1} = T > tj)
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (C[mid] > tj) hi = mid; else lo = mid + 1;
        }
        idx[j] = lo;
    }
}

// New walker j = kept state of walker idx[j] (accept ? proposed : old).
__global__ void k_dmc_gather(int nw, int nc, const int *__restrict__ idx, const uint32_t *__restrict__ accept,
                             qmc_walker_state old, qmc_walker_state prop, qmc_walker_state out, uint64_t *step_ptr)
{
    const int j = blockIdx.x;
    if (j >= nw) return;
    const int k = idx[j];
    const bool a = accept[k] != 0u;
    const qmc_walker_state &src = a ? prop : old;
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        out.R[(size_t)j * nc + c] = src.R[(size_t)k * nc + c];
        out.drift[(size_t)j * nc + c] = src.drift[(size_t)k * nc + c];
    }
    if (threadIdx.x == 0) {
        out.e_loc[j] = src.e_loc[k];
        out.logpsi[j] = src.logpsi[k];
        out.sign[j] = src.sign[k];
        out.status[j] = src.status[k];
        if (j == 0 && step_ptr) *step_ptr += 1;   // every reader of the step ran in an earlier kernel
    }
}

}  // namespace

cudaError_t launch_dmc_move(int nw, int n_elec, const double *R, const double *drift, double tau, uint64_t seed,
                            uint64_t step, const uint64_t *step_ptr, double *Rn, cudaStream_t st)
{
    const int nc = 3 * n_elec;
    const size_t n = (size_t)nw * ((nc + 3) / 4);
    if (n == 0) return cudaSuccess;
    k_dmc_move<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(nw, nc, R, drift, tau, sqrt(tau), seed, step, step_ptr,
                                                           Rn);
    return cudaGetLastError();
}

cudaError_t launch_dmc_weight(int nw, const double *e_old, const double *s_old, const uint32_t *st_old,
                              const double *e_new, const double *s_new, const uint32_t *st_new, double tau,
                              double e_trial, const double *e_trial_ptr, double *weight, uint32_t *accept,
                              cudaStream_t st)
{
    if (nw == 0) return cudaSuccess;
    k_dmc_weight<<<(nw + 255) / 256, 256, 0, st>>>(nw, e_old, s_old, st_old, e_new, s_new, st_new, 0.5 * tau, e_trial,
                                                   e_trial_ptr, weight, accept);
    return cudaGetLastError();
}

cudaError_t launch_srmc(int nw, const double *weight, uint64_t seed, uint64_t step, const uint64_t *step_ptr,
                        unsigned long long *C, int *idx, double *stats, const double *e_new, const double *e_old,
                        const uint32_t *accept, cudaStream_t st)
{
    if (nw == 0) return cudaSuccess;
    k_srmc<<<1, kSrThreads, 0, st>>>(nw, weight, seed, step, step_ptr, C, idx, stats, e_new, e_old, accept);
    return cudaGetLastError();
}

cudaError_t launch_dmc_gather(int nw, int n_elec, const int *idx, const uint32_t *accept, const qmc_walker_state &old,
                              const qmc_walker_state &prop, const qmc_walker_state &out, uint64_t *step_ptr,
                              cudaStream_t st)
{
    if (nw == 0) return cudaSuccess;
    k_dmc_gather<<<nw, 128, 0, st>>>(nw, 3 * n_elec, idx, accept, old, prop, out, step_ptr);
    return cudaGetLastError();
}

}  // namespace qmc
