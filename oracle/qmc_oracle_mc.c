/*
 * qmc_oracle_mc.c -- plain FP64 CPU oracle of the Monte Carlo step around the
 * walker evaluation: the drift-diffusion move, the branching weight and the
 * constant-population reconfiguration (stochastic reconfiguration Monte
 * Carlo, SRMC).
 *
 * TEST INFRASTRUCTURE ONLY, like qmc_oracle.c: only the test-suite, the smoke
 * check and the benchmark's CPU legs load it.  It shares no code, header or
 * constant with the CUDA library.
 *
 * The paper's definitions, in its order (Sec. II.A and II.B):
 *   Eq. (1)  R' = R + tau b(R) + sqrt(tau) eta, eta = 3N independent N(0,1)
 *   Eq. (2)  b = grad Psi_T / Psi_T (from the evaluation)
 *   Eq. (3)  w = exp(-tau/2 [(E_L(R') - E_T) + (E_L(R) - E_T)])
 *   Fixed node (Sec. II.A): the nodes of Psi_T are infinitely repulsive
 *            barriers; a move that would cross one (Psi_T changes sign) is
 *            not made.
 *   Sec. II.B reconfiguration: p_k = w_k / sum_i w_i; M walkers are drawn
 *            among the M walkers with probabilities p_k; the generation's
 *            total weight (sum_i w_i / M) enters the averages through the
 *            product over the preceding generations.
 *
 * Readings where the paper is silent:
 *   - Random numbers: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11), the
 *     counter-based generator, with these streams:
 *       move:  key (seed, 0), counter (j, walker, step, 0): block j gives the
 *              normals 4j..4j+3 of the walker's 3N components (component
 *              3e + c); two Box-Muller pairs (Box and Muller 1958) per block:
 *              u1 = ((x0 >> 11) + 1) 2^-53 in (0, 1], u2 = (x1 >> 11) 2^-53,
 *              n0 = sqrt(-2 ln u1) cos(2 pi u2), n1 = sqrt(-2 ln u1) sin(2 pi u2),
 *              and (x2, x3) -> (n2, n3) the same way;
 *       draws: key (seed, 1), counter (j >> 2, step, 0, 0): output j & 3 is the
 *              64-bit uniform integer U_j of draw j.
 *   - Drawing "according to p_k" is done in exact integer arithmetic so that
 *     the drawn indices are a function of the weights alone: q_k =
 *     floor(2^40 w_k / w_max) (w_k / w_max rounded once, then scaled exactly),
 *     C_k = q_0 + ... + q_k (64-bit integers, exact), t_j = floor(U_j C_{M-1} /
 *     2^64) (the high word of the 128-bit product), and draw j takes the
 *     first k with C_k > t_j.  Walker k is drawn with probability
 *     q_k / C_{M-1} = p_k up to the 2^-40 quantisation.  A weight that is not
 *     finite or not positive counts as 0 (the walker is dropped); if every
 *     weight is 0 the population is kept as it is (idx_j = j).
 *   - A rejected move (sign change, or a proposed walker whose evaluation
 *     failed) keeps the walker at R with its old drift, E_L, log|Psi| and
 *     sign; its weight takes E_L(R') = E_L(R).
 *   - The move is rounded as written: ((R + tau b) + sqrt(tau) eta), with no
 *     fused multiply-add (this file is built with -ffp-contract=off).
 *   - The weight is rounded as exp(-(((E_L' - E_T) + (E_L - E_T)) * (0.5 tau))).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- Philox4x64-10 ------------------------------------------------------ */

static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    const unsigned __int128 p = (unsigned __int128)a * b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

/* One Philox4x64-10 block: ten rounds of the S-box (two 64 x 64 -> 128-bit
 * multiplications, XOR with the other counter words and the round key), the
 * key bumped by the Weyl constants between rounds. */
void oracle_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, c0, &hi0, &lo0);
        mulhilo64(M1, c2, &hi1, &lo1);
        const uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Box-Muller on two 64-bit uniform integers. */
static void box_muller(uint64_t x0, uint64_t x1, double *n0, double *n1)
{
    const double two_pi = 6.283185307179586476925286766559;
    const double u1 = ldexp((double)((x0 >> 11) + 1), -53);
    const double u2 = ldexp((double)(x1 >> 11), -53);
    const double r = sqrt(-2.0 * log(u1));
    const double th = two_pi * u2;
    *n0 = r * cos(th);
    *n1 = r * sin(th);
}

/* The move noise eta[w][q], q = 0..n_comp-1 (n_comp = 3N), of walkers
 * w0..w0+W-1 (stream "move"). */
void oracle_move_normals(int W, int w0, int n_comp, uint64_t seed, uint64_t step, double *eta)
{
    const uint64_t key[2] = {seed, 0};
    for (int w = 0; w < W; ++w)
        for (int j = 0; 4 * j < n_comp; ++j) {
            const uint64_t ctr[4] = {(uint64_t)j, (uint64_t)(w0 + w), step, 0};
            uint64_t x[4];
            double n[4];
            oracle_philox4x64(ctr, key, x);
            box_muller(x[0], x[1], &n[0], &n[1]);
            box_muller(x[2], x[3], &n[2], &n[3]);
            for (int i = 0; i < 4 && 4 * j + i < n_comp; ++i) eta[(size_t)w * n_comp + 4 * j + i] = n[i];
        }
}

/* Eq. (1): R_new = R + tau b + sqrt(tau) eta for W walkers of N electrons. */
void oracle_dmc_move(int W, int N, const double *R, const double *drift, double tau, uint64_t seed, uint64_t step,
                     double *R_new)
{
    const int nc = 3 * N;
    const double st = sqrt(tau);
    double eta[4];
    const uint64_t key[2] = {seed, 0};
    for (int w = 0; w < W; ++w)
        for (int j = 0; 4 * j < nc; ++j) {
            const uint64_t ctr[4] = {(uint64_t)j, (uint64_t)w, step, 0};
            uint64_t x[4];
            oracle_philox4x64(ctr, key, x);
            box_muller(x[0], x[1], &eta[0], &eta[1]);
            box_muller(x[2], x[3], &eta[2], &eta[3]);
            for (int i = 0; i < 4 && 4 * j + i < nc; ++i) {
                const size_t q = (size_t)w * nc + 4 * j + i;
                const double drifted = R[q] + tau * drift[q];
                R_new[q] = drifted + st * eta[i];
            }
        }
}

/* Eq. (3) with the fixed-node rule: accept[w] = 1 if the proposed walker is
 * valid (status_new == 0), the old one was valid and Psi_T kept its sign;
 * the weight uses E_L(R') of the accepted move, else E_L(R) twice.  A walker
 * whose old state is invalid gets weight 0. */
void oracle_dmc_weight(int W, const double *e_old, const double *sign_old, const unsigned *status_old,
                       const double *e_new, const double *sign_new, const unsigned *status_new, double tau,
                       double e_trial, double *weight, unsigned *accept)
{
    for (int w = 0; w < W; ++w) {
        const int valid_old = status_old[w] == 0 && sign_old[w] != 0.0;
        const int acc = valid_old && status_new[w] == 0 && sign_new[w] == sign_old[w];
        accept[w] = (unsigned)acc;
        if (!valid_old) {
            weight[w] = 0.0;
            continue;
        }
        const double en = acc ? e_new[w] : e_old[w];
        const double s = (en - e_trial) + (e_old[w] - e_trial);
        weight[w] = exp(-(s * (0.5 * tau)));
    }
}

/* Sec. II.B: M = W indices drawn with probabilities w_k / sum w (exact
 * integer drawing, above).  wsum[0] = sum of the weights counted (FP64, in
 * walker order), wsum[1] = the number of walkers with a positive finite
 * weight.  Returns 0, or 1 when every weight is 0 (idx = identity). */
int oracle_srmc(int W, const double *weight, uint64_t seed, uint64_t step, int *idx, double *wsum)
{
    double wmax = 0.0, sum = 0.0;
    int alive = 0;
    for (int k = 0; k < W; ++k) {
        const double x = weight[k];
        if (isfinite(x) && x > 0.0) {
            if (x > wmax) wmax = x;
            sum += x;
            ++alive;
        }
    }
    wsum[0] = sum;
    wsum[1] = (double)alive;
    if (!(wmax > 0.0)) {
        for (int j = 0; j < W; ++j) idx[j] = j;
        return 1;
    }
    uint64_t *C = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(W > 0 ? W : 1));
    if (!C) return -1;
    uint64_t acc = 0;
    for (int k = 0; k < W; ++k) {
        const double x = weight[k];
        uint64_t q = 0;
        if (isfinite(x) && x > 0.0) q = (uint64_t)ldexp(x / wmax, 40);
        acc += q;
        C[k] = acc;
    }
    const uint64_t T = acc;
    const uint64_t key[2] = {seed, 1};
    for (int j = 0; j < W; ++j) {
        const uint64_t ctr[4] = {(uint64_t)(j >> 2), step, 0, 0};
        uint64_t x[4];
        oracle_philox4x64(ctr, key, x);
        const uint64_t U = x[j & 3];
        const uint64_t t = (uint64_t)(((unsigned __int128)U * T) >> 64);
        int k = 0;
        while (C[k] <= t) ++k;            /* first k with C_k > t (plain scan) */
        idx[j] = k;
    }
    free(C);
    return 0;
}
