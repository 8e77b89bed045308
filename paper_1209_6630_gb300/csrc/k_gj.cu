// Step a4: log|det|, sign and inverse of each Slater matrix in FP64
// (Sec. II.C: D^-1 for the drift/Laplacian vector products; Sec. IV.B: the
// inversion step, double precision).
//
// One CTA per matrix.  Gauss-Jordan elimination with partial pivoting, done
// in panels of NB = 8, 16 or 32 columns (a tile choice per system):
//   1. the n x NB panel is copied to shared memory and eliminated there,
//      column by column (pivot = largest |entry| among rows not yet used;
//      the pivots are exactly those of LU with partial pivoting);
//   2. every other column j of the matrix receives the panel's row
//      operations at once, as a rank-NB update
//        X[i][j] <- [i not a pivot row] X[i][j] + sum_c P[i][c] X[piv_c][j]
//      (P = the eliminated panel, which holds the composite row operations).
// Pivoting is implicit: rows never move in memory; a row map records which
// physical row was the pivot of each step.  After the last panel the array
// holds Res with X^-1[a][b] = Res[pp[a]][ipp[b]] (pp = pivot rows, ipp its
// inverse), and the kernel writes Dinv = X^-T with a tiled transpose:
//   Dinv[pp[c]][k] = Res[pp[k]][c].
// Flops: n^3 FMA = 2 n^3, the LU (2/3 n^3) plus inverse (4/3 n^3) count.
// Shared memory (n NB + 32 NB) doubles + 3n shorts: at NB = 16, ~75 KB for n = 528
// (three CTAs per SM); NB = 8 halves it at the cost of twice the panel sweeps.
#include <math.h>

#include "ff_math.cuh"
#include "qmc_internal.cuh"

namespace qmc {

constexpr int kGjThreads = 256;
constexpr int kGjWarps = kGjThreads / 32;

struct GjJobs2 {
    GjJob j[2];
};

// doubles reserved for the panel (also holds the 32 x 33 transpose tile)
__host__ __device__ __forceinline__ size_t p_region(int n, int nb)
{
    const size_t a = (size_t)n * nb;
    return a > 32 * 33 ? a : 32 * 33;
}

__device__ __forceinline__ void argmax_merge(double &v, int &i, double v2, int i2)
{
    if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
}

__device__ __forceinline__ void block_argmax(double &bv, int &bi, double *red_v, int *red_i, int lane, int wid)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_down_sync(0xffffffffu, bv, o);
        const int i2 = __shfl_down_sync(0xffffffffu, bi, o);
        argmax_merge(bv, bi, v2, i2);
    }
    if (lane == 0) { red_v[wid] = bv; red_i[wid] = bi; }
}

__device__ __forceinline__ void argmax_merge_f(float &v, int &i, float v2, int i2)
{
    if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
}

__device__ __forceinline__ void block_argmax_f(float &bv, int &bi, float *red_v, int *red_i, int lane, int wid)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float v2 = __shfl_down_sync(0xffffffffu, bv, o);
        const int i2 = __shfl_down_sync(0xffffffffu, bi, o);
        argmax_merge_f(bv, bi, v2, i2);
    }
    if (lane == 0) { red_v[wid] = bv; red_i[wid] = bi; }
}

template <int NB>
__global__ void __launch_bounds__(kGjThreads) k_gj(GjJobs2 jobs)
{
    const GjJob &J = jobs.j[blockIdx.y];
    const int m = blockIdx.x;
    if (m >= J.count) return;
    if (J.only_redo && J.redo[m * J.redo_stride] != 1) return;   // recompute pass: flagged, not yet handled
    const int n = J.n;
    double *__restrict__ X = J.X + (size_t)m * J.x_stride;
    double *__restrict__ Dout = J.Dinv + (size_t)m * J.d_stride;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *P = reinterpret_cast<double *>(smem_raw);   // [n][NB], later a [32][33] tile
    double *U = P + p_region(n, NB);                      // [NB][32]
    short *used = reinterpret_cast<short *>(U + NB * 32); // [n] 1 once a row has been a pivot
    short *pp = used + n;                                 // [n] pivot row of step k
    short *rowc = pp + n;                                 // [n] panel column of a pivot row, or -1
    __shared__ double red_v[kGjWarps];
    __shared__ int red_i[kGjWarps];
    __shared__ int s_p, s_sing;

    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    for (int i = t; i < n; i += kGjThreads) { used[i] = 0; rowc[i] = -1; }
    if (t == 0) s_sing = 0;
    double logabs = 0.0;
    int neg = 0;
    __syncthreads();

    for (int jb = 0; jb < n; jb += NB) {
        const int w = min(NB, n - jb);
        for (int q = t; q < n * NB; q += kGjThreads) {
            const int i = q / NB, c = q - i * NB;
            P[q] = (c < w) ? X[(size_t)i * n + jb + c] : 0.0;
        }
        __syncthreads();
        // pivot candidates of the panel's first column
        double bv = -1.0;
        int bi = n;
        for (int i = t; i < n; i += kGjThreads)
            if (!used[i]) argmax_merge(bv, bi, fabs(P[i * NB]), i);
        block_argmax(bv, bi, red_v, red_i, lane, wid);
        __syncthreads();

        for (int c = 0; c < w; ++c) {
            if (t == 0) {
                double v = red_v[0];
                int b = red_i[0];
                for (int q = 1; q < kGjWarps; ++q) argmax_merge(v, b, red_v[q], red_i[q]);
                s_p = b;
                if (!(v > 0.0)) s_sing = 1;   // exact zero (or NaN) pivot
            }
            __syncthreads();
            if (s_sing) break;
            const int p = s_p;
            const double piv = P[p * NB + c];
            const double inv = 1.0 / piv;
            if (t == 0) {
                used[p] = 1;
                pp[jb + c] = (short)p;
                rowc[p] = (short)c;
                logabs += log(fabs(piv));
                neg ^= (piv < 0.0);
            }
            __syncthreads();   // every thread has read P[p][c] (piv); used[p] is set
            if (t < NB) P[p * NB + t] = (t == c) ? inv : P[p * NB + t] * inv;
            __syncthreads();
            // eliminate column c from the other rows and, on the way, find the
            // pivot candidates of column c+1 among the rows not yet used
            double nbv = -1.0;
            int nbi = n;
            const int cn = c + 1;
            for (int i = t; i < n; i += kGjThreads) {
                if (i == p) continue;
                const double f = P[i * NB + c];
#pragma unroll
                for (int cc = 0; cc < NB; ++cc)
                    if (cc != c) P[i * NB + cc] = fma(-f, P[p * NB + cc], P[i * NB + cc]);
                P[i * NB + c] = -f * inv;
                if (cn < w && !used[i]) argmax_merge(nbv, nbi, fabs(P[i * NB + cn]), i);
            }
            block_argmax(nbv, nbi, red_v, red_i, lane, wid);
            __syncthreads();
        }
        if (s_sing) break;

        // store the eliminated panel
        for (int q = t; q < n * w; q += kGjThreads) {
            const int i = q / w, c = q - i * w;
            X[(size_t)i * n + jb + c] = P[i * NB + c];
        }

        // rank-w update of every other column, 32 columns at a time; the pivot
        // rows of the next chunk are read into registers while this one runs
        int c0 = 0;
        auto skip = [&](int cc0) { return cc0 >= jb && cc0 + 32 <= jb + w; };
        while (c0 < n && skip(c0)) c0 += 32;
        constexpr int UPT = NB * 32 / kGjThreads;   // U elements per thread
        double upre[UPT];
        __syncthreads();   // panel stores done before U reads of the same rows
#pragma unroll
        for (int r = 0; r < UPT; ++r) {
            const int q = t + r * kGjThreads, c = q >> 5, col = c0 + (q & 31);
            upre[r] = (c0 < n && c < w && col < n) ? X[(size_t)pp[jb + c] * n + col] : 0.0;
        }
        while (c0 < n) {
            __syncthreads();   // previous chunk done with U
#pragma unroll
            for (int r = 0; r < UPT; ++r) U[t + r * kGjThreads] = upre[r];
            __syncthreads();
            int c1 = c0 + 32;
            while (c1 < n && skip(c1)) c1 += 32;
#pragma unroll
            for (int r = 0; r < UPT; ++r) {
                const int q = t + r * kGjThreads, c = q >> 5, col = c1 + (q & 31);
                upre[r] = (c1 < n && c < w && col < n) ? X[(size_t)pp[jb + c] * n + col] : 0.0;
            }
            const int col = c0 + lane;
            const bool active = col < n && !(col >= jb && col < jb + w);
            double u[NB];
#pragma unroll
            for (int c = 0; c < NB; ++c) u[c] = U[c * 32 + lane];
            if (active) {
                int i = wid;
                for (; i + 3 * kGjWarps < n; i += 4 * kGjWarps) {
                    double x[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int ii = i + r * kGjWarps;
                        x[r] = (rowc[ii] >= 0) ? 0.0 : X[(size_t)ii * n + col];
                    }
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int ii = i + r * kGjWarps;
                        const double2 *pr = reinterpret_cast<const double2 *>(P + ii * NB);
#pragma unroll
                        for (int c2 = 0; c2 < NB / 2; ++c2) {
                            const double2 pv = pr[c2];
                            x[r] = fma(pv.x, u[2 * c2], x[r]);
                            x[r] = fma(pv.y, u[2 * c2 + 1], x[r]);
                        }
                    }
#pragma unroll
                    for (int r = 0; r < 4; ++r) X[(size_t)(i + r * kGjWarps) * n + col] = x[r];
                }
                for (; i < n; i += kGjWarps) {
                    double x = (rowc[i] >= 0) ? 0.0 : X[(size_t)i * n + col];
                    const double2 *pr = reinterpret_cast<const double2 *>(P + i * NB);
#pragma unroll
                    for (int c2 = 0; c2 < NB / 2; ++c2) {
                        const double2 pv = pr[c2];
                        x = fma(pv.x, u[2 * c2], x);
                        x = fma(pv.y, u[2 * c2 + 1], x);
                    }
                    X[(size_t)i * n + col] = x;
                }
            }
            c0 = c1;
        }
        __syncthreads();
        for (int c = t; c < w; c += kGjThreads) rowc[pp[jb + c]] = -1;
        __syncthreads();
    }

    if (s_sing) {
        const double qnan = __longlong_as_double(0x7ff8000000000000ll);
        for (size_t q = t; q < (size_t)n * n; q += kGjThreads) Dout[q] = qnan;
        if (t == 0) {
            if (J.logabs) J.logabs[(size_t)m * J.la_stride] = -INFINITY;
            if (J.sign) J.sign[(size_t)m * J.la_stride] = 0.0;
            if (J.flag) atomicOr(J.flag + m, J.flag_bit);
        }
        return;
    }
    __syncthreads();   // all panel writes to X visible to the block

    // Dinv[pp[c]][k] = Res[pp[k]][c], 32 x 32 tiles through shared memory
    double *tile = P;   // [32][33]
    for (int kb = 0; kb < n; kb += 32) {
        for (int cb = 0; cb < n; cb += 32) {
            for (int r = wid; r < 32; r += kGjWarps) {
                const int k = kb + r, c = cb + lane;
                tile[r * 33 + lane] = (k < n && c < n) ? X[(size_t)pp[k] * n + c] : 0.0;
            }
            __syncthreads();
            for (int r = wid; r < 32; r += kGjWarps) {
                const int c = cb + r, k = kb + lane;
                if (c < n && k < n) Dout[(size_t)pp[c] * n + k] = tile[lane * 33 + r];
            }
            __syncthreads();
        }
    }

    if (t == 0) {
        // sign of the row permutation k -> pp[k]: parity from its cycles
        int par = 0;
        for (int i = 0; i < n; ++i) used[i] = 0;
        for (int i = 0; i < n; ++i) {
            if (used[i]) continue;
            int len = 0, j = i;
            while (!used[j]) { used[j] = 1; j = pp[j]; ++len; }
            par ^= ((len & 1) == 0);
        }
        if (J.logabs) J.logabs[(size_t)m * J.la_stride] = logabs;
        if (J.sign) J.sign[(size_t)m * J.la_stride] = (par ^ neg) ? -1.0 : 1.0;
    }
}

template <int NB>
static cudaError_t launch_gj_nb(const GjJobs2 &js, int n_jobs, int nmax, int cmax, cudaStream_t st)
{
    const size_t sm = sizeof(double) * (p_region(nmax, NB) + NB * 32) + sizeof(short) * 3 * (size_t)nmax;
    cudaError_t e = cudaFuncSetAttribute(k_gj<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_gj<NB>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    dim3 grid(cmax, n_jobs);
    k_gj<NB><<<grid, kGjThreads, sm, st>>>(js);
    return cudaGetLastError();
}

cudaError_t launch_gj(const GjJob *jobs, int n_jobs, cudaStream_t st, int nb)
{
    GjJobs2 js;
    int nmax = 0, cmax = 0;
    for (int q = 0; q < 2; ++q) {
        js.j[q] = jobs[q < n_jobs ? q : 0];
        if (q >= n_jobs) js.j[q].count = 0;
        nmax = max(nmax, js.j[q].n);
        cmax = max(cmax, js.j[q].count);
    }
    if (cmax == 0) return cudaSuccess;
    switch (nb) {
    case 8: return launch_gj_nb<8>(js, n_jobs, nmax, cmax, st);
    case 16: return launch_gj_nb<16>(js, n_jobs, nmax, cmax, st);
    case 32: return launch_gj_nb<32>(js, n_jobs, nmax, cmax, st);
    default: return cudaErrorInvalidValue;
    }
}


// ---------------------------------------------------------------------------
// Float-float Gauss-Jordan (mixed path, a4 arithmetic QMC_A4_FLOAT_FLOAT).  Same elimination as k_gj, but every
// value is a pair of floats (hi + lo, ~48-bit significand) and the arithmetic
// runs on the FP32 pipes (62x the FP64 rate on this GPU).  The FP64 input X is
// left intact; the elimination works on a float-pair copy.  At the end the
// kernel measures kappa_inf = ||X||_inf ||X^-1||_inf of the result; a matrix
// above `kappa_max` (near a nodal surface of Psi, where the Slater matrix
// becomes singular) or with a non-finite result is flagged, and the caller
// recomputes the flagged matrices with the FP64 k_gj, which skips the others.
// (float-float helpers: ff_math.cuh)

template <int NB>
__global__ void __launch_bounds__(kGjThreads, NB == 8 ? 4 : (NB == 16 ? 3 : 1)) k_gj_ff(GjJobs2 jobs, double kappa_max)
{
    const GjJob &J = jobs.j[blockIdx.y];
    const int m = blockIdx.x;
    if (m >= J.count) return;
    const int n = J.n;
    const double *__restrict__ X = J.X + (size_t)m * J.x_stride;
    float2 *__restrict__ Wk = J.work + (size_t)m * J.x_stride;
    double *__restrict__ Dout = J.Dinv + (size_t)m * J.d_stride;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *P = reinterpret_cast<float2 *>(smem_raw);   // [n][NB], later a [32][33] tile
    float2 *U = P + p_region(n, NB);                      // [NB][32]
    short *used = reinterpret_cast<short *>(U + NB * 32);
    short *pp = used + n;
    short *rowc = pp + n;
    __shared__ int red_i[kGjWarps];
    __shared__ float red_f[kGjWarps];
    __shared__ float s_xnorm;

    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    // float-pair copy of X and ||X||_inf (max row sum of |x|, one warp per row)
    float rmax = 0.f;
    for (int i = wid; i < n; i += kGjWarps) {
        float rs = 0.f;
        for (int c = lane; c < n; c += 32) {
            const double x = X[(size_t)i * n + c];
            const float h = (float)x;
            Wk[(size_t)i * n + c] = make_float2(h, (float)(x - (double)h));
            rs += fabsf(h);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
        rmax = fmaxf(rmax, rs);
    }
    if (lane == 0) red_f[wid] = rmax;
    for (int i = t; i < n; i += kGjThreads) { used[i] = 0; rowc[i] = -1; }
    __syncthreads();
    if (t == 0) {
        float xm = 0.f;
        for (int q = 0; q < kGjWarps; ++q) xm = fmaxf(xm, red_f[q]);
        s_xnorm = xm;
    }
    // |det| = (mag_h + mag_l) 2^mag_e, kept by every thread (the pivots are
    // the same in all threads); the sign from the parity of negative pivots
    float mag_h = 1.f, mag_l = 0.f;
    int mag_e = 0, neg = 0;
    bool sing = false;
    __syncthreads();

    for (int jb = 0; jb < n; jb += NB) {
        const int w = min(NB, n - jb);
        for (int q = t; q < n * NB; q += kGjThreads) {
            const int i = q / NB, c = q - i * NB;
            P[q] = (c < w) ? Wk[(size_t)i * n + jb + c] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        float bv = -1.f;
        int bi = n;
        for (int i = t; i < n; i += kGjThreads)
            if (!used[i]) argmax_merge_f(bv, bi, fabsf(P[i * NB].x), i);
        block_argmax_f(bv, bi, red_f, red_i, lane, wid);
        __syncthreads();

        // NB consecutive lanes share a row, one panel column each: the
        // accesses of a warp are contiguous (no bank conflicts)
        const int cc = t & (NB - 1);
        for (int c = 0; c < w; ++c) {
            // every thread merges the warps' candidates in the same order
            float v = red_f[0];
            int p = red_i[0];
            for (int q = 1; q < kGjWarps; ++q) argmax_merge_f(v, p, red_f[q], red_i[q]);
            if (!(v > 0.f)) { sing = true; break; }
            const float2 piv = P[p * NB + c];
            const float2 pinv = ff::inv(piv);
            const float2 prow = (cc == c) ? pinv : ff::mul(P[p * NB + cc], pinv);
            {
                const float2 a = piv.x < 0.f ? ff::neg(piv) : piv;
                const float2 mg = ff::mul(make_float2(mag_h, mag_l), a);
                int ex;
                frexpf(mg.x, &ex);
                mag_h = ldexpf(mg.x, -ex);
                mag_l = ldexpf(mg.y, -ex);
                mag_e += ex;
                neg ^= piv.x < 0.f;
            }
            if (t == 0) {
                used[p] = 1;
                pp[jb + c] = (short)p;
                rowc[p] = (short)c;
            }
            __syncthreads();                               // the candidates and row p have been read
            if (t < NB) P[p * NB + t] = prow;              // t < NB: column cc == t
            float nbv = -1.f;
            int nbi = n;
            const int cn = c + 1;
            for (int base = (t & ~31) / NB; base < n; base += kGjThreads / NB) {
                const int i = base + lane / NB;
                const bool live = i < n && i != p;
                const float2 mf = live ? ff::neg(P[i * NB + c]) : make_float2(0.f, 0.f);
                __syncwarp();                              // every lane has read P[i][c]
                if (live) {
                    const float2 x = (cc != c) ? ff::fma2(P[i * NB + cc], mf, prow) : ff::mul(mf, pinv);
                    P[i * NB + cc] = x;
                    if (cc == cn && cn < w && !used[i]) argmax_merge_f(nbv, nbi, fabsf(x.x), i);
                }
            }
            block_argmax_f(nbv, nbi, red_f, red_i, lane, wid);
            __syncthreads();
        }
        if (sing) break;

        for (int q = t; q < n * w; q += kGjThreads) {
            const int i = q / w, c = q - i * w;
            Wk[(size_t)i * n + jb + c] = P[i * NB + c];
        }

        int c0 = 0;
        auto skip = [&](int cc0) { return cc0 >= jb && cc0 + 32 <= jb + w; };
        while (c0 < n && skip(c0)) c0 += 32;
        constexpr int UPT = NB * 32 / kGjThreads;
        float2 upre[UPT];
        __syncthreads();
#pragma unroll
        for (int r = 0; r < UPT; ++r) {
            const int q = t + r * kGjThreads, c = q >> 5, col = c0 + (q & 31);
            upre[r] = (c0 < n && c < w && col < n) ? Wk[(size_t)pp[jb + c] * n + col] : make_float2(0.f, 0.f);
        }
        while (c0 < n) {
            __syncthreads();
#pragma unroll
            for (int r = 0; r < UPT; ++r) U[t + r * kGjThreads] = upre[r];
            __syncthreads();
            int c1 = c0 + 32;
            while (c1 < n && skip(c1)) c1 += 32;
#pragma unroll
            for (int r = 0; r < UPT; ++r) {
                const int q = t + r * kGjThreads, c = q >> 5, col = c1 + (q & 31);
                upre[r] = (c1 < n && c < w && col < n) ? Wk[(size_t)pp[jb + c] * n + col] : make_float2(0.f, 0.f);
            }
            const int col = c0 + lane;
            const bool active = col < n && !(col >= jb && col < jb + w);
            float2 u[NB];
#pragma unroll
            for (int c = 0; c < NB; ++c) u[c] = U[c * 32 + lane];
            if (active) {
                // rows (i, i + 8) two iterations ahead are loaded while the
                // current pair is updated
                auto load_pair = [&](int i, float2 &a, float2 &b) {
                    const int i2 = i + kGjWarps;
                    a = (i < n && rowc[i] < 0) ? Wk[(size_t)i * n + col] : make_float2(0.f, 0.f);
                    b = (i2 < n && rowc[i2] < 0) ? Wk[(size_t)i2 * n + col] : make_float2(0.f, 0.f);
                };
                float2 nx0, nx1, mx0, mx1;                 // two row pairs ahead
                load_pair(wid, nx0, nx1);
                load_pair(wid + 2 * kGjWarps, mx0, mx1);
#pragma unroll 2
                for (int i = wid; i < n; i += 2 * kGjWarps) {
                    // two rows at a time; products of a row summed with TwoSum
                    // into the hi part and plain FP32 into the lo part, one
                    // renormalisation per row at the end
                    const int i2 = i + kGjWarps;
                    const bool has2 = i2 < n;
                    float2 x0 = nx0, x1 = nx1;
                    nx0 = mx0;
                    nx1 = mx1;
                    load_pair(i + 4 * kGjWarps, mx0, mx1);
                    const float4 *pr0 = reinterpret_cast<const float4 *>(P + i * NB);
                    const float4 *pr1 = reinterpret_cast<const float4 *>(P + (has2 ? i2 : i) * NB);
#pragma unroll
                    for (int c2 = 0; c2 < NB / 2; ++c2) {
                        const float4 a0 = pr0[c2], a1 = pr1[c2];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const float2 uv = u[2 * c2 + h];
                            const float ph0 = h ? a0.z : a0.x, pl0 = h ? a0.w : a0.y;
                            const float ph1 = h ? a1.z : a1.x, pl1 = h ? a1.w : a1.y;
                            float p = __fmul_rn(ph0, uv.x), pe = fmaf(ph0, uv.x, -p);
                            pe = fmaf(ph0, uv.y, pe);
                            pe = fmaf(pl0, uv.x, pe);
                            float s, e;
                            ff::two_sum(x0.x, p, s, e);
                            x0.x = s;
                            x0.y = __fadd_rn(x0.y, __fadd_rn(pe, e));
                            p = __fmul_rn(ph1, uv.x);
                            pe = fmaf(ph1, uv.x, -p);
                            pe = fmaf(ph1, uv.y, pe);
                            pe = fmaf(pl1, uv.x, pe);
                            ff::two_sum(x1.x, p, s, e);
                            x1.x = s;
                            x1.y = __fadd_rn(x1.y, __fadd_rn(pe, e));
                        }
                    }
                    float h0, l0;
                    ff::fast_two_sum(x0.x, x0.y, h0, l0);
                    Wk[(size_t)i * n + col] = make_float2(h0, l0);
                    if (has2) {
                        ff::fast_two_sum(x1.x, x1.y, h0, l0);
                        Wk[(size_t)i2 * n + col] = make_float2(h0, l0);
                    }
                }
            }
            c0 = c1;
        }
        __syncthreads();
        for (int c = t; c < w; c += kGjThreads) rowc[pp[jb + c]] = -1;
        __syncthreads();
    }

    if (sing) {
        // a zero pivot in the float pairs: the FP64 kernel decides whether X is singular
        if (t == 0 && J.redo) J.redo[m * J.redo_stride] = 1;
        return;
    }
    __syncthreads();

    // ||X^-1||_inf: the rows of X^-1 are the rows of the result (columns permuted)
    float imax = 0.f;
    for (int i = wid; i < n; i += kGjWarps) {
        float rs = 0.f;
        for (int c = lane; c < n; c += 32) rs += fabsf(Wk[(size_t)i * n + c].x);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
        imax = fmaxf(imax, rs);
    }
    if (lane == 0) red_f[wid] = imax;

    float2 *tile = P;   // [32][33]
    for (int kb = 0; kb < n; kb += 32) {
        for (int cb = 0; cb < n; cb += 32) {
            for (int r = wid; r < 32; r += kGjWarps) {
                const int k = kb + r, c = cb + lane;
                tile[r * 33 + lane] = (k < n && c < n) ? Wk[(size_t)pp[k] * n + c] : make_float2(0.f, 0.f);
            }
            __syncthreads();
            for (int r = wid; r < 32; r += kGjWarps) {
                const int c = cb + r, k = kb + lane;
                if (c < n && k < n) Dout[(size_t)pp[c] * n + k] = ff::val(tile[lane * 33 + r]);
            }
            __syncthreads();
        }
    }

    if (t == 0) {
        float im = 0.f;
        for (int q = 0; q < kGjWarps; ++q) im = fmaxf(im, red_f[q]);
        const double kappa = (double)s_xnorm * (double)im;
        int par = 0;
        for (int i = 0; i < n; ++i) used[i] = 0;
        for (int i = 0; i < n; ++i) {
            if (used[i]) continue;
            int len = 0, j = i;
            while (!used[j]) { used[j] = 1; j = pp[j]; ++len; }
            par ^= ((len & 1) == 0);
        }
        const double logabs = log((double)mag_h + (double)mag_l) + mag_e * 0.69314718055994530942;
        if (J.logabs) J.logabs[(size_t)m * J.la_stride] = logabs;
        if (J.sign) J.sign[(size_t)m * J.la_stride] = (par ^ neg) ? -1.0 : 1.0;
        if (J.redo && !(kappa <= kappa_max && isfinite(logabs))) J.redo[m * J.redo_stride] = 1;
    }
}

template <int NB>
static cudaError_t launch_gj_ff_nb(const GjJobs2 &js, int n_jobs, int nmax, int cmax, double kappa_max,
                                   cudaStream_t st)
{
    const size_t sm = sizeof(float2) * (p_region(nmax, NB) + NB * 32) + sizeof(short) * 3 * (size_t)nmax;
    cudaError_t e = cudaFuncSetAttribute(k_gj_ff<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_gj_ff<NB>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    dim3 grid(cmax, n_jobs);
    k_gj_ff<NB><<<grid, kGjThreads, sm, st>>>(js, kappa_max);
    return cudaGetLastError();
}

cudaError_t launch_gj_ff(const GjJob *jobs, int n_jobs, cudaStream_t st, int nb, double kappa_max)
{
    GjJobs2 js;
    int nmax = 0, cmax = 0;
    for (int q = 0; q < 2; ++q) {
        js.j[q] = jobs[q < n_jobs ? q : 0];
        if (q >= n_jobs) js.j[q].count = 0;
        nmax = max(nmax, js.j[q].n);
        cmax = max(cmax, js.j[q].count);
    }
    if (cmax == 0) return cudaSuccess;
    switch (nb) {
    case 8: return launch_gj_ff_nb<8>(js, n_jobs, nmax, cmax, kappa_max, st);
    case 16: return launch_gj_ff_nb<16>(js, n_jobs, nmax, cmax, kappa_max, st);
    case 32: return launch_gj_ff_nb<32>(js, n_jobs, nmax, cmax, kappa_max, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace qmc
