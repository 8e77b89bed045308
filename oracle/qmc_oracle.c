/*
 * qmc_oracle.c -- plain, slow, FP64 CPU oracle of the all-electron walker
 * evaluation (Slater matrices from localized atomic Gaussians).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header
 * or constant with the CUDA library; it reads the same seeded inputs.
 *
 * Every step follows the paper's definitions in the paper's order:
 *   Sec. II.C, Eq. (mo)          phi_i(r) = sum_j a_ij chi_j(r)
 *   Sec. II.C, AO form / Eq. (Gaussian)
 *                                chi(r) = (x-Qx)^nx (y-Qy)^ny (z-Qz)^nz g(r),
 *                                g(r) = sum_k c_k exp(-gamma_k |r-Q|^2)
 *   Sec. II.C, Slater matrix     D_ij = phi_i(r_j), derivative matrices D^(1), D^(2)
 *   Sec. II.C, drift/Laplacian   (1/Det) dDet/dx_l^i = sum_j (D^-1)_ij d_l phi_j(r_i)
 *                                (indices read as the standard identity; the
 *                                printed formula is garbled)
 *   Sec. III, screening          AO, gradient, Laplacian are zero where g < eps;
 *                                an atomic radius gives an early exit
 *   Sec. III, Eq. (abc) and the practical product loop: for each electron,
 *                                for each non-zero AO (ascending), for each MO,
 *                                accumulate the five products C1..C5
 *   Eq. (2) drift b = grad Psi / Psi, Eq. (4) local energy E_L = H Psi / Psi
 *   Sec. IV.B inversion step     LU with partial pivoting, log|det|, inverse
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fno-fast-math -shared -fPIC
 * (no FMA contraction: the screening distance must be rounded exactly as
 * written, d2 = ((dx*dx) + (dy*dy)) + (dz*dz)).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int n_atom;
    const double *Z;          /* [n_atom] */
    const double *Q;          /* [n_atom][3] */
    int n_shell;
    const int *shell_atom;    /* [n_shell] */
    const int *shell_L;
    const int *shell_nprim;
    const int *shell_pstart;
    const double *prim_gamma; /* [n_prim] */
    const double *prim_coef;
    int n_ao;
    const int *ao_shell;      /* [n_ao] */
    const int *ao_pow;        /* [n_ao][3] */
    const double *ao_scale;   /* [n_ao] */
    int n_up, n_dn;
    const double *A_up;       /* [n_ao][n_up]  row = AO, column = MO */
    const double *A_dn;       /* [n_ao][n_dn] */
    double eps;
    const double *R2;         /* [n_shell] screening radii^2 (from oracle_shell_r2) */
    int unscreened;           /* 1: every AO active (no screening) */
    const int *sh_ao0;        /* [n_shell] first AO of each shell (oracle_shell_ranges) */
    const int *sh_nao;        /* [n_shell] number of AOs of each shell */
    /* Jastrow factor e^J (Sec. II.C, the J of Eq. psit), off unless jas_on:
     * J = sum_{i<j} U_ee(r_ij) + sum_i sum_a U_en(r_ia),
     * U_ee(r) = a r / (1 + b_ee r) with a = ja_par (same spins) or ja_anti,
     * U_en(r) = -ja_en[a] r / (1 + jb_en[a] r).                          */
    int jas_on;
    double ja_par, ja_anti, jb_ee;
    const double *ja_en;      /* [n_atom] */
    const double *jb_en;      /* [n_atom] */
} osys;

/* AOs are stored shell by shell; record each shell's contiguous AO range. */
int oracle_shell_ranges(const osys *s, int *sh_ao0, int *sh_nao)
{
    for (int t = 0; t < s->n_shell; ++t) { sh_ao0[t] = -1; sh_nao[t] = 0; }
    for (int mu = 0; mu < s->n_ao; ++mu) {
        int t = s->ao_shell[mu];
        if (sh_ao0[t] < 0) sh_ao0[t] = mu;
        else if (sh_ao0[t] + sh_nao[t] != mu) return -1;   /* not contiguous */
        sh_nao[t] += 1;
    }
    return 0;
}

enum { ST_SINGULAR_UP = 1u, ST_SINGULAR_DN = 2u, ST_NONFINITE = 4u };

/* ------------------------------------------------------------------ */
/* Sec. III: radius of a shell.  g(x) = sum_k c_k exp(-gamma_k x) with
 * x = |r-Q|^2.  R2 is the smallest non-negative double x with g(x) < eps,
 * located by bisection on the IEEE-754 bit patterns of non-negative doubles
 * (monotone for non-negative values).  An AO is kept iff d2 < R2.          */
static double shell_g(const osys *s, int sh, double x)
{
    double g = 0.0;
    int p0 = s->shell_pstart[sh];
    for (int k = 0; k < s->shell_nprim[sh]; ++k)
        g = g + s->prim_coef[p0 + k] * exp(-s->prim_gamma[p0 + k] * x);
    return g;
}

static int64_t dbits(double x) { int64_t b; memcpy(&b, &x, 8); return b; }
static double bitsd(int64_t b) { double x; memcpy(&x, &b, 8); return x; }

void oracle_shell_r2(const osys *s, double *R2)
{
    for (int sh = 0; sh < s->n_shell; ++sh) {
        if (shell_g(s, sh, 0.0) < s->eps) { R2[sh] = 0.0; continue; }
        double hi = 1.0;
        while (!(shell_g(s, sh, hi) < s->eps)) hi = hi * 2.0;
        int64_t lo_b = dbits(0.0), hi_b = dbits(hi);
        while (hi_b - lo_b > 1) {
            int64_t mid = lo_b + (hi_b - lo_b) / 2;
            if (shell_g(s, sh, bitsd(mid)) < s->eps) hi_b = mid; else lo_b = mid;
        }
        R2[sh] = bitsd(hi_b);
    }
}

/* ------------------------------------------------------------------ */
/* Sec. III: per-electron list of non-zero AOs (ascending AO index).     */
static double sqdist(const double *r, const double *q)
{
    double dx = r[0] - q[0], dy = r[1] - q[1], dz = r[2] - q[2];
    double xx = dx * dx, yy = dy * dy, zz = dz * dz;
    return (xx + yy) + zz;
}

int oracle_screen(const osys *s, const double *r, int *idx, int cap)
{
    int K = 0;
    int sh = 0;
    for (int a = 0; a < s->n_atom; ++a) {
        int sh_end = sh;
        while (sh_end < s->n_shell && s->shell_atom[sh_end] == a) ++sh_end;
        double d2 = sqdist(r, &s->Q[3 * a]);
        double ratom = 0.0;       /* atomic radius^2 = max over its shells */
        for (int t = sh; t < sh_end; ++t) if (s->R2[t] > ratom) ratom = s->R2[t];
        if (s->unscreened || d2 < ratom) {
            for (int t = sh; t < sh_end; ++t) {
                if (!s->unscreened && !(d2 < s->R2[t])) continue;
                for (int m = 0; m < s->sh_nao[t]; ++m) {   /* AOs of shell t, ascending */
                    if (K < cap) idx[K] = s->sh_ao0[t] + m;
                    ++K;
                }
            }
        }
        sh = sh_end;
    }
    return K;
}

/* ------------------------------------------------------------------ */
/* Sec. II.C AO form: value, gradient and Laplacian of chi_mu at r.
 * out[0]=chi, out[1..3]=d chi/dx,dy,dz, out[4]=Laplacian.             */
static double ipow(double x, int n)
{
    double p = 1.0;
    for (int i = 0; i < n; ++i) p = p * x;
    return p;
}

void oracle_ao(const osys *s, const double *r, int mu, double *out)
{
    int sh = s->ao_shell[mu];
    int a = s->shell_atom[sh];
    const double *q = &s->Q[3 * a];
    double d[3] = { r[0] - q[0], r[1] - q[1], r[2] - q[2] };
    double d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
    int n[3] = { s->ao_pow[3 * mu], s->ao_pow[3 * mu + 1], s->ao_pow[3 * mu + 2] };

    /* radial part g and its derivatives: grad g = -2 d sum c_k gamma_k e_k,
     * lap g = sum c_k (4 gamma_k^2 d2 - 6 gamma_k) e_k                     */
    double g = 0.0, gd = 0.0, gl = 0.0;
    int p0 = s->shell_pstart[sh];
    for (int k = 0; k < s->shell_nprim[sh]; ++k) {
        double gam = s->prim_gamma[p0 + k], c = s->prim_coef[p0 + k];
        double e = exp(-gam * d2);
        g += c * e;
        gd += c * gam * e;
        gl += c * (4.0 * gam * gam * d2 - 6.0 * gam) * e;
    }
    double grad_g[3] = { -2.0 * d[0] * gd, -2.0 * d[1] * gd, -2.0 * d[2] * gd };

    /* polynomial part P = dx^nx dy^ny dz^nz and its derivatives */
    double P = ipow(d[0], n[0]) * ipow(d[1], n[1]) * ipow(d[2], n[2]);
    double dP[3], d2P[3];
    for (int l = 0; l < 3; ++l) {
        double others = 1.0;
        for (int m = 0; m < 3; ++m) if (m != l) others *= ipow(d[m], n[m]);
        dP[l] = (n[l] >= 1) ? n[l] * ipow(d[l], n[l] - 1) * others : 0.0;
        d2P[l] = (n[l] >= 2) ? n[l] * (n[l] - 1) * ipow(d[l], n[l] - 2) * others : 0.0;
    }
    double sc = s->ao_scale[mu];
    out[0] = sc * P * g;
    for (int l = 0; l < 3; ++l) out[1 + l] = sc * (dP[l] * g + P * grad_g[l]);
    double lapP = d2P[0] + d2P[1] + d2P[2];
    double dPdg = dP[0] * grad_g[0] + dP[1] * grad_g[1] + dP[2] * grad_g[2];
    out[4] = sc * (lapP * g + 2.0 * dPdg + P * gl);
}

/* ------------------------------------------------------------------ */
/* Sec. III practical algorithm: for electron i, non-zero AO k (ascending),
 * MO j:  C_l(j,i) += A(j, indices(k,i)) * B_l(k,i).  C_l is stored
 * electron-major, C[l][i][j] = d_l phi_j(r_i) (l=0 value, 1..3 gradient,
 * 4 Laplacian).  A(j,mu) is the MO coefficient a_{j mu} = A_s[mu][j].     */
static void slater(const osys *s, int spin, const double *R /* [N][3] */,
                   int cap, int *idx, double *B, double *C /* [5][ns][ns] */,
                   int *cnt_out, int *idx_out, double *B_out)
{
    int ns = spin ? s->n_dn : s->n_up;
    int e0 = spin ? s->n_up : 0;
    const double *A = spin ? s->A_dn : s->A_up;
    memset(C, 0, sizeof(double) * 5 * (size_t)ns * ns);
    for (int i = 0; i < ns; ++i) {
        const double *r = &R[3 * (e0 + i)];
        int K = oracle_screen(s, r, idx, cap);
        if (K > cap) K = cap;      /* caller sizes cap = n_ao, so never hit */
        for (int k = 0; k < K; ++k) oracle_ao(s, r, idx[k], &B[5 * k]);
        if (cnt_out) cnt_out[e0 + i] = K;
        if (idx_out) for (int k = 0; k < K; ++k) idx_out[(size_t)(e0 + i) * cap + k] = idx[k];
        if (B_out) for (int k = 0; k < K; ++k) for (int l = 0; l < 5; ++l)
            B_out[((size_t)(e0 + i) * 5 + l) * cap + k] = B[5 * k + l];
        for (int k = 0; k < K; ++k) {
            const double *arow = &A[(size_t)idx[k] * ns];
            for (int j = 0; j < ns; ++j) {
                double a = arow[j];
                for (int l = 0; l < 5; ++l)
                    C[((size_t)l * ns + i) * ns + j] += a * B[5 * k + l];
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* Sec. IV.B inversion step: LU with partial pivoting (pivot = first row
 * attaining max |a|), log|det| = sum log|u_ii|, sign from the row
 * interchanges and the signs of u_ii; inverse by forward and backward
 * substitution on the columns of the identity.  M is n x n row-major and is
 * overwritten by its LU factors.  Returns 1 if an exact zero pivot occurs.  */
int oracle_lu_inverse(int n, double *M, double *logabs, double *sign, double *Minv)
{
    int *perm = (int *)malloc(sizeof(int) * n);
    double *col = (double *)malloc(sizeof(double) * n);
    for (int i = 0; i < n; ++i) perm[i] = i;
    double la = 0.0, sg = 1.0;
    int singular = 0;
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(M[(size_t)k * n + k]);
        for (int i = k + 1; i < n; ++i) {
            double v = fabs(M[(size_t)i * n + k]);
            if (v > best) { best = v; p = i; }
        }
        if (p != k) {
            for (int j = 0; j < n; ++j) {
                double t = M[(size_t)k * n + j];
                M[(size_t)k * n + j] = M[(size_t)p * n + j];
                M[(size_t)p * n + j] = t;
            }
            int t = perm[k]; perm[k] = perm[p]; perm[p] = t;
            sg = -sg;
        }
        double piv = M[(size_t)k * n + k];
        if (piv == 0.0) { singular = 1; break; }
        la += log(fabs(piv));
        if (piv < 0.0) sg = -sg;
        for (int i = k + 1; i < n; ++i) {
            double f = M[(size_t)i * n + k] / piv;
            M[(size_t)i * n + k] = f;
            for (int j = k + 1; j < n; ++j)
                M[(size_t)i * n + j] -= f * M[(size_t)k * n + j];
        }
    }
    if (singular) {
        *logabs = -INFINITY; *sign = 0.0;
        free(perm); free(col);
        return 1;
    }
    *logabs = la; *sign = sg;
    if (Minv) {
        /* column c of M^-1 solves L U x = P e_c */
        for (int c = 0; c < n; ++c) {
            for (int i = 0; i < n; ++i) col[i] = (perm[i] == c) ? 1.0 : 0.0;
            for (int i = 0; i < n; ++i) {               /* L y = P e_c */
                double v = col[i];
                for (int j = 0; j < i; ++j) v -= M[(size_t)i * n + j] * col[j];
                col[i] = v;
            }
            for (int i = n - 1; i >= 0; --i) {          /* U x = y */
                double v = col[i];
                for (int j = i + 1; j < n; ++j) v -= M[(size_t)i * n + j] * col[j];
                col[i] = v / M[(size_t)i * n + i];
            }
            for (int i = 0; i < n; ++i) Minv[(size_t)i * n + c] = col[i];
        }
    }
    free(perm); free(col);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Coulomb terms of the all-electron Born-Oppenheimer Hamiltonian.        */
double oracle_vnn(const osys *s)
{
    double v = 0.0;
    for (int a = 0; a < s->n_atom; ++a)
        for (int b = a + 1; b < s->n_atom; ++b) {
            double dx = s->Q[3 * a] - s->Q[3 * b], dy = s->Q[3 * a + 1] - s->Q[3 * b + 1],
                   dz = s->Q[3 * a + 2] - s->Q[3 * b + 2];
            v += s->Z[a] * s->Z[b] / sqrt(dx * dx + dy * dy + dz * dz);
        }
    return v;
}

static double v_en(const osys *s, const double *R, int N)
{
    double v = 0.0;
    for (int i = 0; i < N; ++i)
        for (int a = 0; a < s->n_atom; ++a) {
            double dx = R[3 * i] - s->Q[3 * a], dy = R[3 * i + 1] - s->Q[3 * a + 1],
                   dz = R[3 * i + 2] - s->Q[3 * a + 2];
            v -= s->Z[a] / sqrt(dx * dx + dy * dy + dz * dz);
        }
    return v;
}

static double v_ee(const double *R, int N)
{
    double v = 0.0;
    for (int i = 0; i < N; ++i)
        for (int j = i + 1; j < N; ++j) {
            double dx = R[3 * i] - R[3 * j], dy = R[3 * i + 1] - R[3 * j + 1],
                   dz = R[3 * i + 2] - R[3 * j + 2];
            v += 1.0 / sqrt(dx * dx + dy * dy + dz * dz);
        }
    return v;
}

/* ------------------------------------------------------------------ */
/* The Jastrow factor of one walker: J, and per electron its gradient g_i =
 * grad_i J and Laplacian L_i = lap_i J.  Pade form U(r) = a r / (1 + b r):
 * U' = a / (1 + b r)^2, U'' = -2 a b / (1 + b r)^3, lap_i U(|r_i - x|) =
 * U'' + 2 U' / r, grad_i U = U' (r_i - x) / r.  Pairs in natural order.    */
static double jastrow(const osys *s, const double *R, int N, double *g /*[N][3]*/, double *L /*[N]*/)
{
    double J = 0.0;
    for (int i = 0; i < 3 * N; ++i) g[i] = 0.0;
    for (int i = 0; i < N; ++i) L[i] = 0.0;
    for (int i = 0; i < N; ++i)
        for (int j = i + 1; j < N; ++j) {
            const double a = ((i < s->n_up) == (j < s->n_up)) ? s->ja_par : s->ja_anti, b = s->jb_ee;
            double d[3];
            for (int l = 0; l < 3; ++l) d[l] = R[3 * i + l] - R[3 * j + l];
            const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            const double q = 1.0 + b * r;
            const double u = a * r / q, u1 = a / (q * q), u2 = -2.0 * a * b / (q * q * q);
            J += u;
            for (int l = 0; l < 3; ++l) {
                g[3 * i + l] += u1 * d[l] / r;
                g[3 * j + l] -= u1 * d[l] / r;
            }
            L[i] += u2 + 2.0 * u1 / r;
            L[j] += u2 + 2.0 * u1 / r;
        }
    for (int i = 0; i < N; ++i)
        for (int at = 0; at < s->n_atom; ++at) {
            const double a = -s->ja_en[at], b = s->jb_en[at];
            double d[3];
            for (int l = 0; l < 3; ++l) d[l] = R[3 * i + l] - s->Q[3 * at + l];
            const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            const double q = 1.0 + b * r;
            const double u = a * r / q, u1 = a / (q * q), u2 = -2.0 * a * b / (q * q * q);
            J += u;
            for (int l = 0; l < 3; ++l) g[3 * i + l] += u1 * d[l] / r;
            L[i] += u2 + 2.0 * u1 / r;
        }
    return J;
}

/* ------------------------------------------------------------------ */
/* One walker, full evaluation.  Outputs:
 *   logabs[2], sgn[2] per spin; drift[N][3]; parts[4] = T, V_en, V_ee, V_nn;
 *   e_loc; dinv (optional) [n_up*n_up + n_dn*n_dn], D^-1 of each spin with
 *   rows = electrons, columns = MOs;  optional debug dumps.               */
typedef struct {
    int cap;
    int *cnt;        /* [N] */
    int *idx;        /* [N][cap] */
    double *B;       /* [N][5][cap] */
    double *C;       /* [5][n_up][n_up] then [5][n_dn][n_dn] */
} odebug;

static unsigned eval_one(const osys *s, const double *R, double vnn,
                         double *logabs, double *sgn, double *drift, double *parts,
                         double *e_loc, double *dinv, const odebug *dbg, double *jas_out)
{
    int N = s->n_up + s->n_dn;
    unsigned status = 0;
    int cap = s->n_ao;
    int *idx = (int *)malloc(sizeof(int) * cap);
    double *B = (double *)malloc(sizeof(double) * 5 * cap);
    double T = 0.0;
    for (int i = 0; i < 3 * N; ++i) if (!isfinite(R[i])) status |= ST_NONFINITE;
    size_t doff = 0;
    for (int spin = 0; spin < 2; ++spin) {
        int ns = spin ? s->n_dn : s->n_up;
        int e0 = spin ? s->n_up : 0;
        double *C = (double *)malloc(sizeof(double) * 5 * (size_t)ns * ns);
        double *D = (double *)malloc(sizeof(double) * (size_t)ns * ns);
        double *Dinv = (double *)malloc(sizeof(double) * (size_t)ns * ns);
        slater(s, spin, R, cap, idx, B, C,
               dbg ? dbg->cnt : NULL, dbg ? dbg->idx : NULL, dbg ? dbg->B : NULL);
        if (dbg && dbg->C) {
            size_t off = spin ? 5 * (size_t)s->n_up * s->n_up : 0;
            memcpy(dbg->C + off, C, sizeof(double) * 5 * (size_t)ns * ns);
        }
        /* Slater matrix D_ji = phi_j(r_i): row j = MO, column i = electron */
        for (int j = 0; j < ns; ++j)
            for (int i = 0; i < ns; ++i) D[(size_t)j * ns + i] = C[(size_t)i * ns + j];
        int sing = oracle_lu_inverse(ns, D, &logabs[spin], &sgn[spin], Dinv);
        if (sing) {
            status |= spin ? ST_SINGULAR_DN : ST_SINGULAR_UP;
            for (int i = 0; i < ns; ++i) for (int l = 0; l < 3; ++l) drift[3 * (e0 + i) + l] = NAN;
            T = NAN;
        } else {
            /* drift and Laplacian of electron i: sum_j (D^-1)_ij d_l phi_j(r_i) */
            for (int i = 0; i < ns; ++i) {
                double b[4] = { 0.0, 0.0, 0.0, 0.0 };
                for (int j = 0; j < ns; ++j) {
                    double w = Dinv[(size_t)i * ns + j];
                    for (int l = 0; l < 4; ++l) b[l] += w * C[((size_t)(1 + l) * ns + i) * ns + j];
                }
                for (int l = 0; l < 3; ++l) drift[3 * (e0 + i) + l] = b[l];
                T += -0.5 * b[3];
            }
        }
        if (dinv) {
            for (size_t t = 0; t < (size_t)ns * ns; ++t) dinv[doff + t] = sing ? NAN : Dinv[t];
        }
        doff += (size_t)ns * ns;
        free(C); free(D); free(Dinv);
    }
    /* Jastrow: Psi = e^J Det_up Det_dn, so grad_i Psi / Psi = g_i + b_i and
     * lap_i Psi / Psi = L_i + |g_i|^2 + 2 g_i . b_i + lap_i Det / Det        */
    double J = 0.0;
    if (s->jas_on) {
        double *g = (double *)malloc(sizeof(double) * 3 * (size_t)N);
        double *L = (double *)malloc(sizeof(double) * (size_t)N);
        J = jastrow(s, R, N, g, L);
        for (int i = 0; i < N; ++i) {
            double gb = 0.0, gg = 0.0;
            for (int l = 0; l < 3; ++l) {
                gg += g[3 * i + l] * g[3 * i + l];
                gb += g[3 * i + l] * drift[3 * i + l];
            }
            T += -0.5 * (L[i] + gg + 2.0 * gb);
            for (int l = 0; l < 3; ++l) drift[3 * i + l] += g[3 * i + l];
        }
        free(g); free(L);
    }
    if (jas_out) *jas_out = J;
    double ven = v_en(s, R, N), vee = v_ee(R, N);
    parts[0] = T; parts[1] = ven; parts[2] = vee; parts[3] = vnn;
    *e_loc = T + ven + vee + vnn;
    if (!(status & (ST_SINGULAR_UP | ST_SINGULAR_DN))) {
        if (!isfinite(*e_loc) || !isfinite(logabs[0]) || !isfinite(logabs[1])) status |= ST_NONFINITE;
    }
    free(idx); free(B);
    return status;
}

/* Batch evaluation; walkers in parallel (OpenMP, dynamic schedule). */
int oracle_eval(const osys *s, int W, const double *R, int nthreads,
                double *logpsi, double *sign, double *logabs /*[W][2]*/, double *drift,
                double *e_loc, double *e_parts, unsigned *status, double *dinv)
{
    int N = s->n_up + s->n_dn;
    double vnn = oracle_vnn(s);
    size_t dsz = (size_t)s->n_up * s->n_up + (size_t)s->n_dn * s->n_dn;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int w = 0; w < W; ++w) {
        double la[2], sg[2], J;
        unsigned st = eval_one(s, &R[(size_t)w * 3 * N], vnn, la, sg, &drift[(size_t)w * 3 * N],
                               &e_parts[4 * (size_t)w], &e_loc[w], dinv ? &dinv[w * dsz] : NULL, NULL, &J);
        logabs[2 * w] = la[0]; logabs[2 * w + 1] = la[1];
        logpsi[w] = la[0] + la[1] + J;
        sign[w] = sg[0] * sg[1];
        status[w] = st;
    }
    return 0;
}

int oracle_eval_debug(const osys *s, const double *R, int cap, int *cnt, int *idx, double *B,
                      double *C, double *logabs, double *sgn, double *drift, double *parts,
                      double *e_loc, double *dinv, unsigned *status, double *jas)
{
    odebug dbg = { cap, cnt, idx, B, C };
    if (cap < s->n_ao) return -1;
    *status = eval_one(s, R, oracle_vnn(s), logabs, sgn, drift, parts, e_loc, dinv, &dbg, jas);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Adjoint: d log|Psi| / d a_{j mu} = sum_i (D^-1)_ij chi_mu(r_i) (derived
 * from the same cofactor identity as the drift).  Weighted over walkers:
 * dA_s[mu][j] = sum_w g_w sum_{i in s} (D^-1)_w,ij chi_mu(r_w,i), with the
 * screened chi (the function being differentiated is the screened one).   */
int oracle_logpsi_grad(const osys *s, int W, const double *R, const double *g, int nthreads,
                       double *dA_up, double *dA_dn)
{
    int N = s->n_up + s->n_dn;
    int nao = s->n_ao;
    memset(dA_up, 0, sizeof(double) * (size_t)nao * s->n_up);
    memset(dA_dn, 0, sizeof(double) * (size_t)nao * s->n_dn);
    double vnn = oracle_vnn(s);
    size_t dsz = (size_t)s->n_up * s->n_up + (size_t)s->n_dn * s->n_dn;
    int nt = 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    nt = omp_get_max_threads();
#endif
    double *part_up = (double *)calloc((size_t)nt * nao * s->n_up, sizeof(double));
    double *part_dn = (double *)calloc((size_t)nt * nao * s->n_dn, sizeof(double));
#ifdef _OPENMP
#pragma omp parallel
#endif
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        double *dinv = (double *)malloc(sizeof(double) * dsz);
        double *drift = (double *)malloc(sizeof(double) * 3 * N);
        int *idx = (int *)malloc(sizeof(int) * nao);
        double chi[5];
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int w = 0; w < W; ++w) {
            double la[2], sg[2], parts[4], el;
            const double *Rw = &R[(size_t)w * 3 * N];
            eval_one(s, Rw, vnn, la, sg, drift, parts, &el, dinv, NULL, NULL);
            size_t doff = 0;
            for (int spin = 0; spin < 2; ++spin) {
                int ns = spin ? s->n_dn : s->n_up;
                int e0 = spin ? s->n_up : 0;
                double *G = spin ? &part_dn[(size_t)t * nao * ns] : &part_up[(size_t)t * nao * ns];
                for (int i = 0; i < ns; ++i) {
                    const double *r = &Rw[3 * (e0 + i)];
                    int K = oracle_screen(s, r, idx, nao);
                    for (int k = 0; k < K; ++k) {
                        int mu = idx[k];
                        oracle_ao(s, r, mu, chi);
                        double f = g[w] * chi[0];
                        for (int j = 0; j < ns; ++j)
                            G[(size_t)mu * ns + j] += f * dinv[doff + (size_t)i * ns + j];
                    }
                }
                doff += (size_t)ns * ns;
            }
        }
        free(dinv); free(drift); free(idx);
    }
    for (int t = 0; t < nt; ++t) {
        for (size_t q = 0; q < (size_t)nao * s->n_up; ++q) dA_up[q] += part_up[(size_t)t * nao * s->n_up + q];
        for (size_t q = 0; q < (size_t)nao * s->n_dn; ++q) dA_dn[q] += part_dn[(size_t)t * nao * s->n_dn + q];
    }
    free(part_up); free(part_dn);
    return 0;
}

/* Single AO at arbitrary points (for derivative and normalisation pins). */
void oracle_ao_points(const osys *s, int mu, int npt, const double *r, double *out /*[npt][5]*/)
{
    for (int p = 0; p < npt; ++p) oracle_ao(s, &r[3 * p], mu, &out[5 * p]);
}

int oracle_screen_points(const osys *s, int npt, const double *r, int cap, int *cnt, int *idx)
{
    for (int p = 0; p < npt; ++p) cnt[p] = oracle_screen(s, &r[3 * p], &idx[(size_t)p * cap], cap);
    return 0;
}
