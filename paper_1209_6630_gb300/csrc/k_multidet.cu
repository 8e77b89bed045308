// Multi-determinant trial function (Sec. II.C, Eq. psit):
//   Psi = e^J sum_K c_K Det_K,up Det_K,dn = sum_K c_K Psi_K,
// combined from the evaluations of the single determinants Psi_K (each a
// loaded system with its own MO coefficients, the same nuclei, basis and
// Jastrow factor).  With L_K = log|Psi_K|, s_K its sign, L = max L_K over the
// determinants that are not singular, S = sum_K c_K s_K e^{L_K - L} and the
// weights w_K = c_K s_K e^{L_K - L} / S (sum_K w_K = 1):
//   log|Psi| = L + log|S|,  sign = sign(S),
//   drift = grad Psi / Psi = sum_K w_K b_K,
//   lap Psi / Psi = sum_K w_K (lap Psi_K / Psi_K), so T and E_L are the same
//   weighted sums (the potential does not depend on K).
// One CTA per walker: thread 0 forms the weights, all threads combine the drift.
#include <math.h>

#include "qmc_internal.cuh"

namespace qmc {

namespace {

constexpr int kMdThreads = 128;

struct MdCoef {
    double c[kMaxDets];
};

__global__ void __launch_bounds__(kMdThreads) k_multidet_combine(int nw, int N, int K, MdCoef cf,
                                                                 const double *__restrict__ lp,   // [K][nw]
                                                                 const double *__restrict__ sg,   // [K][nw]
                                                                 const double *__restrict__ dr,   // [K][nw][N][3]
                                                                 const double *__restrict__ el,   // [K][nw]
                                                                 const double *__restrict__ ep,   // [K][nw][4]
                                                                 const uint32_t *__restrict__ st, // [K][nw]
                                                                 qmc_eval_out o)
{
    __shared__ double wk[kMaxDets];
    __shared__ int s_bad;
    const int w = blockIdx.x;
    if (w >= nw) return;
    if (threadIdx.x == 0) {
        double L = -INFINITY;
        for (int k = 0; k < K; ++k) {
            const double l = lp[(size_t)k * nw + w], s = sg[(size_t)k * nw + w];
            const bool live = s != 0.0 && isfinite(l) && !(st[(size_t)k * nw + w] & QMC_STATUS_NONFINITE);
            if (live && l > L) L = l;
        }
        double S = 0.0;
        for (int k = 0; k < K; ++k) {
            const double l = lp[(size_t)k * nw + w], s = sg[(size_t)k * nw + w];
            const bool live = s != 0.0 && isfinite(l) && !(st[(size_t)k * nw + w] & QMC_STATUS_NONFINITE);
            wk[k] = live ? cf.c[k] * s * exp(l - L) : 0.0;
            S += wk[k];
        }
        uint32_t status = 0;
        for (int k = 0; k < K; ++k) status |= st[(size_t)k * nw + w] & QMC_STATUS_TIMEOUT;
        const bool sing = !(S != 0.0) || !isfinite(L);
        s_bad = sing;
        if (sing) {
            status |= QMC_STATUS_SINGULAR_UP | QMC_STATUS_SINGULAR_DN;
            o.logpsi[w] = -INFINITY;
            o.sign[w] = 0.0;
            o.e_loc[w] = NAN;
            if (o.e_parts) for (int q = 0; q < 4; ++q) o.e_parts[4 * (size_t)w + q] = NAN;
        } else {
            double e = 0.0, T = 0.0;
            for (int k = 0; k < K; ++k) {
                wk[k] /= S;
                if (wk[k] != 0.0) {
                    e += wk[k] * el[(size_t)k * nw + w];
                    T += wk[k] * ep[((size_t)k * nw + w) * 4];
                }
            }
            o.logpsi[w] = L + log(fabs(S));
            o.sign[w] = S > 0.0 ? 1.0 : -1.0;
            o.e_loc[w] = e;
            if (o.e_parts) {
                o.e_parts[4 * (size_t)w] = T;
                for (int q = 1; q < 4; ++q) o.e_parts[4 * (size_t)w + q] = ep[(size_t)w * 4 + q];   // the same V for all K
            }
            if (!isfinite(e) || !isfinite(o.logpsi[w])) status |= QMC_STATUS_NONFINITE;
        }
        if (o.logabs) { o.logabs[2 * (size_t)w] = NAN; o.logabs[2 * (size_t)w + 1] = NAN; }
        o.status[w] = status;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < 3 * N; c += kMdThreads) {
        double x = NAN;
        if (!s_bad) {
            x = 0.0;
            for (int k = 0; k < K; ++k)
                if (wk[k] != 0.0) x += wk[k] * dr[((size_t)k * nw + w) * 3 * N + c];
        }
        o.drift[(size_t)w * 3 * N + c] = x;
    }
}

}  // namespace

cudaError_t launch_multidet_combine(int nw, int N, int K, const double *coef, const double *lp, const double *sg,
                                    const double *dr, const double *el, const double *ep, const uint32_t *st,
                                    const qmc_eval_out &o, cudaStream_t stream)
{
    if (nw == 0) return cudaSuccess;
    if (K < 1 || K > kMaxDets) return cudaErrorInvalidValue;
    MdCoef cf;
    for (int k = 0; k < K; ++k) cf.c[k] = coef[k];      // host coefficients, passed by value
    k_multidet_combine<<<nw, kMdThreads, 0, stream>>>(nw, N, K, cf, lp, sg, dr, el, ep, st, o);
    return cudaGetLastError();
}

}  // namespace qmc
