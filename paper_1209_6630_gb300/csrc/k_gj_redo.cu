// Step a4, mixed path: FP64 recomputation of the matrices that the
// float-float Gauss-Jordan pass flagged (near a nodal surface of Psi, where
// the Slater matrix approaches singularity; Sec. IV.B keeps the inversion in
// double precision).
//
// A 528 x 528 FP64 elimination on one SM is bound by that SM's FP64 pipe
// (~35 ms), so a single flagged matrix would dominate the stage.  Here each
// flagged matrix is spread over many CTAs: for every panel of NB columns one
// CTA eliminates the panel (partial pivoting among rows not yet used; the
// same arithmetic, order and panel width as k_gj, so the results are
// identical) and then one CTA per 32-column block applies the rank-NB update
// to its columns,
//   X[i][j] <- [i not a pivot of the panel] X[i][j] + sum_c P[i][c] X[piv_c][j],
// two launches per panel.  Grids are fixed (kRedoMax matrices); a list kernel
// collects the flagged matrices in a deterministic order and marks them
// handled (flag 2); flagged matrices beyond the list keep flag 1 and go
// through k_gj.  With nothing flagged every CTA exits at once.
#include <math.h>

#include "qmc_device.cuh"

namespace qmc {

constexpr int kRThreads = 256;
constexpr int kRWarps = kRThreads / 32;

struct RedoEntry {
    int job, m;
};

struct RedoList {
    int count;
    RedoEntry e[kRedoMax];
};

// per listed matrix: logabs, negative-pivot parity, singular flag, pivot rows
// pp[n] and the panel in which each row became a pivot (-1: not yet)
struct RedoState {
    double logabs;
    int neg, sing;
};

struct RedoArgs {
    GjJob j[2];
    RedoList *list;
    char *state;           // kRedoMax entries of state_stride bytes
    size_t state_stride;
    int nmax;
    int e_off[2];          // first electron of each job's spin
};

__device__ __forceinline__ RedoState *rstate(const RedoArgs &a, int b)
{
    return reinterpret_cast<RedoState *>(a.state + (size_t)b * a.state_stride);
}
__device__ __forceinline__ short *rpp(const RedoArgs &a, int b)
{
    return reinterpret_cast<short *>(a.state + (size_t)b * a.state_stride + 16);
}
__device__ __forceinline__ short *rpanel(const RedoArgs &a, int b)
{
    return rpp(a, b) + a.nmax;
}

size_t redo_scratch_bytes(int nmax)
{
    const size_t stride = (16 + 4 * (size_t)nmax + 255) & ~size_t(255);
    return ((sizeof(RedoList) + 255) & ~size_t(255)) + kRedoMax * stride;
}

__device__ __forceinline__ void rargmax(double &v, int &i, double v2, int i2)
{
    if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
}

__device__ __forceinline__ void rblock_argmax(double &bv, int &bi, double *red_v, int *red_i, int lane, int wid)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_down_sync(0xffffffffu, bv, o);
        const int i2 = __shfl_down_sync(0xffffffffu, bi, o);
        rargmax(bv, bi, v2, i2);
    }
    if (lane == 0) { red_v[wid] = bv; red_i[wid] = bi; }
}

// Collect flagged matrices (flag 1) of both jobs, job 0 first, in index order.
__global__ void __launch_bounds__(1024) k_redo_list(RedoArgs a, int n_jobs)
{
    __shared__ int warp_s[32];
    __shared__ int s_base;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    if (t == 0) s_base = 0;
    __syncthreads();
    for (int job = 0; job < n_jobs; ++job) {
        const GjJob &J = a.j[job];
        for (int m0 = 0; m0 < J.count; m0 += 1024) {
            const int m = m0 + t;
            const int f = (m < J.count && J.redo[(size_t)m * J.redo_stride] == 1) ? 1 : 0;
            int x = f;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) warp_s[wid] = x;
            __syncthreads();
            int before = 0, total = 0;
            for (int q = 0; q < 32; ++q) {
                if (q < wid) before += warp_s[q];
                total += warp_s[q];
            }
            const int pos = s_base + before + x - f;
            if (f && pos < kRedoMax) {
                a.list->e[pos].job = job;
                a.list->e[pos].m = m;
                J.redo[(size_t)m * J.redo_stride] = 2;
            }
            __syncthreads();
            if (t == 0) s_base += total;
            __syncthreads();
        }
    }
    if (t == 0) a.list->count = min(s_base, kRedoMax);
}

// Eliminate panel [jb, jb + w) of every listed matrix (one CTA each).
template <int kRNB>
__global__ void __launch_bounds__(kRThreads) k_redo_panel(RedoArgs a, int jb)
{
    const int b = blockIdx.x;
    if (b >= a.list->count) return;
    const RedoEntry en = a.list->e[b];
    const GjJob &J = a.j[en.job];
    const int n = J.n;
    if (jb >= n) return;
    RedoState *stt = rstate(a, b);
    short *pp = rpp(a, b), *panel = rpanel(a, b);
    double *__restrict__ X = J.X + (size_t)en.m * J.x_stride;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *P = reinterpret_cast<double *>(smem_raw);             // [n][kRNB]
    short *used = reinterpret_cast<short *>(P + (size_t)n * kRNB);  // [n]
    __shared__ double red_v[kRWarps];
    __shared__ int red_i[kRWarps];
    __shared__ int s_p, s_sing;
    __shared__ double s_logabs;
    __shared__ int s_neg;

    if (jb == 0) {
        for (int i = t; i < n; i += kRThreads) panel[i] = -1;
        if (t == 0) { stt->logabs = 0.0; stt->neg = 0; stt->sing = 0; }
        __syncthreads();
    }
    if (t == 0) { s_sing = stt->sing; s_logabs = stt->logabs; s_neg = stt->neg; }
    __syncthreads();
    if (s_sing) return;
    const int w = min(kRNB, n - jb);
    for (int i = t; i < n; i += kRThreads) used[i] = panel[i] >= 0;
    for (int q = t; q < n * kRNB; q += kRThreads) {
        const int i = q / kRNB, c = q - i * kRNB;
        P[q] = (c < w) ? X[(size_t)i * n + jb + c] : 0.0;
    }
    __syncthreads();
    double bv = -1.0;
    int bi = n;
    for (int i = t; i < n; i += kRThreads)
        if (!used[i]) rargmax(bv, bi, fabs(P[i * kRNB]), i);
    rblock_argmax(bv, bi, red_v, red_i, lane, wid);
    __syncthreads();
    for (int c = 0; c < w; ++c) {
        if (t == 0) {
            double v = red_v[0];
            int p = red_i[0];
            for (int q = 1; q < kRWarps; ++q) rargmax(v, p, red_v[q], red_i[q]);
            s_p = p;
            if (!(v > 0.0)) s_sing = 1;
        }
        __syncthreads();
        if (s_sing) break;
        const int p = s_p;
        const double piv = P[p * kRNB + c];
        const double inv = 1.0 / piv;
        if (t == 0) {
            used[p] = 1;
            pp[jb + c] = (short)p;
            panel[p] = (short)jb;
            s_logabs += log(fabs(piv));
            s_neg ^= (piv < 0.0);
        }
        __syncthreads();
        if (t < kRNB) P[p * kRNB + t] = (t == c) ? inv : P[p * kRNB + t] * inv;
        __syncthreads();
        double nbv = -1.0;
        int nbi = n;
        const int cn = c + 1;
        for (int i = t; i < n; i += kRThreads) {
            if (i == p) continue;
            const double f = P[i * kRNB + c];
#pragma unroll
            for (int cc = 0; cc < kRNB; ++cc)
                if (cc != c) P[i * kRNB + cc] = fma(-f, P[p * kRNB + cc], P[i * kRNB + cc]);
            P[i * kRNB + c] = -f * inv;
            if (cn < w && !used[i]) rargmax(nbv, nbi, fabs(P[i * kRNB + cn]), i);
        }
        rblock_argmax(nbv, nbi, red_v, red_i, lane, wid);
        __syncthreads();
    }
    if (!s_sing)
        for (int q = t; q < n * w; q += kRThreads) {
            const int i = q / w, c = q - i * w;
            X[(size_t)i * n + jb + c] = P[i * kRNB + c];
        }
    if (t == 0) { stt->sing = s_sing; stt->logabs = s_logabs; stt->neg = s_neg; }
}

// Rank-w update of the 32 columns of block blockIdx.x of every listed matrix.
template <int kRNB>
__global__ void __launch_bounds__(kRThreads) k_redo_update(RedoArgs a, int jb)
{
    const int b = blockIdx.y;
    if (b >= a.list->count) return;
    const RedoEntry en = a.list->e[b];
    const GjJob &J = a.j[en.job];
    const int n = J.n;
    const int c0 = blockIdx.x * 32;
    if (jb >= n || c0 >= n) return;
    const int w = min(kRNB, n - jb);
    if (c0 >= jb && c0 + 32 <= jb + w) return;            // entirely inside the panel
    const RedoState *stt = rstate(a, b);
    if (stt->sing) return;
    const short *pp = rpp(a, b), *panel = rpanel(a, b);
    double *__restrict__ X = J.X + (size_t)en.m * J.x_stride;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *P = reinterpret_cast<double *>(smem_raw);   // [n][kRNB]
    double *U = P + (size_t)n * kRNB;                    // [kRNB][32]
    for (int q = t; q < n * kRNB; q += kRThreads) {
        const int i = q / kRNB, c = q - i * kRNB;
        P[q] = (c < w) ? X[(size_t)i * n + jb + c] : 0.0;
    }
    for (int q = t; q < kRNB * 32; q += kRThreads) {
        const int c = q >> 5, col = c0 + (q & 31);
        U[q] = (c < w && col < n) ? X[(size_t)pp[jb + c] * n + col] : 0.0;
    }
    __syncthreads();
    const int col = c0 + lane;
    if (col >= n || (col >= jb && col < jb + w)) return;
    double u[kRNB];
#pragma unroll
    for (int c = 0; c < kRNB; ++c) u[c] = U[c * 32 + lane];
    for (int i = wid; i < n; i += kRWarps) {
        double x = (panel[i] == jb) ? 0.0 : X[(size_t)i * n + col];
        const double2 *pr = reinterpret_cast<const double2 *>(P + i * kRNB);
#pragma unroll
        for (int c2 = 0; c2 < kRNB / 2; ++c2) {
            const double2 pv = pr[c2];
            x = fma(pv.x, u[2 * c2], x);
            x = fma(pv.y, u[2 * c2 + 1], x);
        }
        X[(size_t)i * n + col] = x;
    }
}

// D^-1, log|det| and sign of every listed matrix: Dinv[pp[c]][k] = Res[pp[k]][c].
__global__ void __launch_bounds__(kRThreads) k_redo_final(RedoArgs a)
{
    const int b = blockIdx.x;
    if (b >= a.list->count) return;
    const RedoEntry en = a.list->e[b];
    const GjJob &J = a.j[en.job];
    const int n = J.n, m = en.m;
    const RedoState *stt = rstate(a, b);
    const short *pp = rpp(a, b);
    const double *__restrict__ X = J.X + (size_t)m * J.x_stride;
    double *__restrict__ Dout = J.Dinv + (size_t)m * J.d_stride;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    __shared__ double tile[32 * 33];
    __shared__ unsigned char seen[1024];
    if (stt->sing) {
        const double qnan = __longlong_as_double(0x7ff8000000000000ll);
        for (size_t q = t; q < (size_t)n * n; q += kRThreads) Dout[q] = qnan;
        if (t == 0) {
            if (J.logabs) J.logabs[(size_t)m * J.la_stride] = -INFINITY;
            if (J.sign) J.sign[(size_t)m * J.la_stride] = 0.0;
            if (J.flag) atomicOr(J.flag + m, J.flag_bit);
        }
        return;
    }
    for (int kb = 0; kb < n; kb += 32)
        for (int cb = 0; cb < n; cb += 32) {
            for (int r = wid; r < 32; r += kRWarps) {
                const int k = kb + r, c = cb + lane;
                tile[r * 33 + lane] = (k < n && c < n) ? X[(size_t)pp[k] * n + c] : 0.0;
            }
            __syncthreads();
            for (int r = wid; r < 32; r += kRWarps) {
                const int c = cb + r, k = kb + lane;
                if (c < n && k < n) Dout[(size_t)pp[c] * n + k] = tile[lane * 33 + r];
            }
            __syncthreads();
        }
    if (t == 0) {
        int par = 0;
        for (int i = 0; i < n; ++i) seen[i] = 0;
        for (int i = 0; i < n; ++i) {
            if (seen[i]) continue;
            int len = 0, j = i;
            while (!seen[j]) { seen[j] = 1; j = pp[j]; ++len; }
            par ^= ((len & 1) == 0);
        }
        if (J.logabs) J.logabs[(size_t)m * J.la_stride] = stt->logabs;
        if (J.sign) J.sign[(size_t)m * J.la_stride] = (par ^ stt->neg) ? -1.0 : 1.0;
    }
}

// C1 rows of every listed matrix recomputed in FP64 (exact screening, FP64 AO
// values and products): near a nodal surface the mixed-precision C1 (~2^-40
// normwise) perturbs log|det| by up to kappa times that.  Each CTA computes
// one row (blockIdx.x) of every 32nd listed matrix; thread t owns MO columns
// t, t + 128, ...
constexpr int kC1Threads = 128;
constexpr int kC1Chunk = 512;

__device__ __forceinline__ void redo_c1_row(const SysDev &s, const RedoArgs &a, const double *__restrict__ R, int b)
{
    const RedoEntry en = a.list->e[b];
    const GjJob &J = a.j[en.job];
    const int n = J.n, i = blockIdx.x;
    if (i >= n) return;
    const int e = a.e_off[en.job] + i;
    const int spin = e >= s.n_up;
    const double *__restrict__ A = s.A64[spin];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *b_s = reinterpret_cast<double *>(smem_raw);             // [kC1Chunk]
    int *idx_s = reinterpret_cast<int *>(b_s + kC1Chunk);            // [n_ao]
    __shared__ int warp_s[kC1Threads / 32];
    const double *r = R + ((size_t)en.m * s.n_elec + e) * 3;
    const double rx = r[0], ry = r[1], rz = r[2];
    const int K = screen_electron<kC1Threads>(s, rx, ry, rz, idx_s, s.n_ao, warp_s);
    double *__restrict__ Xrow = J.X + (size_t)en.m * J.x_stride + (size_t)i * n;
    constexpr int kMaxCols = 1024 / kC1Threads;
    double acc[kMaxCols];
#pragma unroll
    for (int j = 0; j < kMaxCols; ++j) acc[j] = 0.0;
    for (int k0 = 0; k0 < K; k0 += kC1Chunk) {
        const int kc = min(kC1Chunk, K - k0);
        for (int q = threadIdx.x; q < kc; q += kC1Threads) b_s[q] = ao_value_f64(s, idx_s[k0 + q], rx, ry, rz);
        __syncthreads();
        for (int q = 0; q < kc; ++q) {
            const double bv = b_s[q];
            const double *Arow = A + (size_t)idx_s[k0 + q] * n;
#pragma unroll
            for (int j = 0; j < kMaxCols; ++j) {
                const int k = threadIdx.x + kC1Threads * j;
                if (k < n) acc[j] = fma(bv, Arow[k], acc[j]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < kMaxCols; ++j) {
        const int k = threadIdx.x + kC1Threads * j;
        if (k < n) Xrow[k] = acc[j];
    }
}

constexpr int kC1Slots = 32;   // CTAs per row; each loops over the listed matrices

__global__ void __launch_bounds__(kC1Threads) k_redo_c1(SysDev s, RedoArgs a, const double *__restrict__ R)
{
    for (int b = blockIdx.y; b < a.list->count; b += kC1Slots) redo_c1_row(s, a, R, b);
}

template <int NB>
static cudaError_t launch_redo_panels(const RedoArgs &a, int nmax, cudaStream_t st)
{
    const size_t smp = sizeof(double) * (size_t)nmax * NB + sizeof(short) * nmax;
    const size_t smu = sizeof(double) * ((size_t)nmax * NB + NB * 32);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_redo_panel<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smp)) !=
        cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_redo_update<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smu)) !=
        cudaSuccess)
        return e;
    const dim3 ugrid((nmax + 31) / 32, kRedoMax);
    for (int jb = 0; jb < nmax; jb += NB) {
        k_redo_panel<NB><<<kRedoMax, kRThreads, smp, st>>>(a, jb);
        k_redo_update<NB><<<ugrid, kRThreads, smu, st>>>(a, jb);
    }
    return cudaGetLastError();
}

// nb: panel width, the same as the FP64 k_gj of this system (identical results).
// With R given, the listed matrices' C1 is first recomputed in FP64 from the
// walkers' positions (e_off: first electron of each job's spin).
cudaError_t launch_gj_redo(const GjJob *jobs, int n_jobs, void *scratch, cudaStream_t st, int nb, const SysDev *s,
                           const double *R, const int *e_off)
{
    RedoArgs a;
    int nmax = 0;
    for (int q = 0; q < 2; ++q) {
        a.j[q] = jobs[q < n_jobs ? q : 0];
        if (q >= n_jobs) a.j[q].count = 0;
        nmax = max(nmax, a.j[q].n);
    }
    if (n_jobs == 0 || nmax == 0) return cudaSuccess;
    if (nmax > 1024) return cudaErrorInvalidValue;
    a.nmax = nmax;
    a.list = static_cast<RedoList *>(scratch);
    a.state = static_cast<char *>(scratch) + ((sizeof(RedoList) + 255) & ~size_t(255));
    a.state_stride = (16 + 4 * (size_t)nmax + 255) & ~size_t(255);
    a.e_off[0] = e_off ? e_off[0] : 0;
    a.e_off[1] = e_off ? e_off[1] : 0;
    k_redo_list<<<1, 1024, 0, st>>>(a, n_jobs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (R && s) {
        const size_t sm = sizeof(double) * kC1Chunk + sizeof(int) * (size_t)s->n_ao;
        if ((e = cudaFuncSetAttribute(k_redo_c1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess)
            return e;
        k_redo_c1<<<dim3(nmax, kC1Slots), kC1Threads, sm, st>>>(*s, a, R);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    switch (nb) {
    case 8: e = launch_redo_panels<8>(a, nmax, st); break;
    case 16: e = launch_redo_panels<16>(a, nmax, st); break;
    case 32: e = launch_redo_panels<32>(a, nmax, st); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    k_redo_final<<<kRedoMax, kRThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace qmc
