// Step a4 of the mixed path with the panel updates on the tcgen05 tensor
// cores (a4 arithmetic QMC_A4_TENSOR).
//
// The Gauss-Jordan elimination with partial pivoting of k_gj / k_gj_ff
// (implicit pivoting: rows never move, a row map records the pivots; after
// the last panel the array holds Res with X^-1[a][b] = Res[pp[a]][ipp[b]]),
// on a float-pair work matrix (~48-bit significand), in panels of kGtB = 32
// columns, as launches over all matrices of a walker chunk:
//
//   k_gt_init    float-pair copy of X (rows padded to an even length) and ||X||_inf
//   per panel jb:
//   k_gt_panel_t one CTA per matrix eliminates the n x 32 panel in shared
//   (k_gt_panel) memory (pivot = the first row with the largest |entry| among
//                the rows not used yet: the pivots of LU with partial
//                pivoting) -- one thread per row, in sub-panels of 8 with
//                rank-8 updates between them, up to 544 rows, else one warp
//                per row -- and writes the operands of the panel's update in
//                exact BF16 slices: the panel P [n][32] (row i scaled by
//                2^-E_i) and the pivot rows U [32][n] as they were before the
//                update (column j scaled by 2^-F_j), seven slices of 7 bits
//                each (the scheme of the C1/C5 products, one slice more)
//   k_gt_update  X[i][j] <- [i is not a pivot row of the panel] X[i][j]
//                           + sum_c P[i][c] U[c][j]
//                for every column j outside the panel; one CTA per 128 rows,
//                warp-specialised (warps moving the old values by tensor TMA
//                and the operands by bulk copies, an MMA warp, 16 epilogue
//                warps), loops over
//                the 32-column tiles and issues, per tile, 2 K16
//                steps x 28 slice-pair MMAs into seven TMEM
//                accumulators, one per order d = i + j <= 6 of the pair: each
//                sums at most 7 x 32 products of at most 128 x 128 units of
//                2^-7(d+2), below 2^24 units, so every kept product is added
//                exactly; the dropped orders d >= 7 are below ~2^-47 of the
//                update (float pairs: 2^-48).  The epilogue adds orders 0..3
//                as float pairs and 4..6 (below 2^-21 of the update) first in
//                FP32 (rounding ~2^-46), scales by 2^(E_i + F_j) as two exact
//                FP32 multiplications and adds the result to the float-pair X
//   k_gt_final   ||X^-1||_inf, kappa_inf, log|det| and its sign, D^-1 = X^-T
//
// Matrices with kappa_inf above the threshold, a zero pivot, a non-finite
// result or an expired bounded wait are flagged, and the FP64 recomputation
// (C1 from the positions and the FP64 elimination) replaces them, exactly as
// for k_gj_ff.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "ff_math.cuh"
#include "qmc_internal.cuh"
#include "slices.cuh"
#include "umma.cuh"

namespace qmc {

constexpr int kGtB = 32;                             // panel width = K of the update
constexpr int kGtThreads = 256;                      // init and final kernels
constexpr int kGtWarps = kGtThreads / 32;
constexpr int kGpThreads = 512;                      // panel kernel: one warp per row, 16 rows at a time
constexpr int kGpWarps = kGpThreads / 32;
constexpr int kGtEpWarps = 16;                       // update kernel: 4 lane quadrants x 4 groups of 8 columns,
constexpr int kGtUpThreads = 32 * (kGtEpWarps + 3);  // plus the X, B and MMA warps
constexpr int kGtN = 32;                             // columns per update tile (= the panel width)
constexpr int kGtSl = 7;                             // slices per operand
constexpr uint32_t kGtAPlane = 128 * kGtB * 2;       // [128 rows][32 K] BF16, K-major, 64-byte swizzle: 8 KB
constexpr uint32_t kGtBPlane = kGtB * kGtN * 2;      // [32 K][32 columns] BF16, MN-major, 64-byte swizzle: 2 KB
constexpr uint32_t kGtBSbo = 512;                    // next group of 8 K rows (one 32-column atom each)
constexpr int kGtBs = 3;                             // stages of pivot-row slices
constexpr int kGtXs = 3;                             // stages of old values
constexpr uint32_t kGtXStage = 128 * kGtN * 8;       // [2 halves][128 rows][16 float pairs], 128-byte swizzle
constexpr uint32_t kGtATmem = 256;                   // TMEM: 7 accumulators of 32 columns at 0, the panel
                                                     // slices (7 x 16 columns) from 256

// MN-major, 64-byte swizzle, one 32-column atom per group of 8 K rows: byte
// offset of the 16-byte chunk holding columns n0..n0+7 of K row r
__device__ __forceinline__ uint32_t b_off32c(int r, int n0)
{
    return (uint32_t)((r >> 3) * kGtBSbo + (r & 7) * 64 + ((((n0 & 31) >> 3) ^ ((r & 7) >> 1)) << 4));
}

struct GtState {                                     // per matrix, kept across the panel launches
    float mag_h, mag_l;                              // |det| = (mag_h + mag_l) 2^mag_e
    int mag_e, neg, sing;
    float xnorm;                                     // ||X||_inf
    int pad[2];
};

struct GtLayout {                                    // scratch of one matrix
    size_t w, a, b, e, f, pp, used, piv, state, per;
};

__host__ __device__ inline size_t gt_al(size_t x) { return (x + 255) & ~(size_t)255; }

// row stride of the float-pair work matrix: n rounded up to even, so that every row and
// every 32-column segment of it starts on a 16-byte boundary (the bulk copies' rule)
__host__ __device__ inline int gt_ld(int n) { return (n + 1) & ~1; }

__host__ __device__ inline GtLayout gt_layout(int n)
{
    const size_t nt = (size_t)(n + 127) / 128, nc = (size_t)(n + kGtN - 1) / kGtN;
    GtLayout L;
    size_t o = 0;
    L.w = o; o += gt_al(8 * (size_t)n * gt_ld(n));     // the float-pair work matrix [n][gt_ld(n)]
    L.a = o; o += nt * kGtSl * kGtAPlane;             // [row tile][slice] planes of P
    L.b = o; o += nc * kGtSl * kGtBPlane;             // [column tile][slice] planes of U
    L.e = o; o += gt_al(4 * nt * 128);                // E_i
    L.f = o; o += gt_al(4 * nt * 128);                // F_j
    L.pp = o; o += gt_al(2 * (size_t)n);              // pivot row of each column
    L.used = o; o += gt_al(2 * (size_t)n);            // row already a pivot
    L.piv = o; o += gt_al((size_t)n);                 // row is a pivot of the current panel
    L.state = o; o += 256;
    L.per = gt_al(o);
    return L;
}

struct GtJobs {
    GjJob j[2];
    unsigned char *scr[2];                           // scratch of matrix m: scr + m * per
    int nj;
    int jb;                                          // current panel
    unsigned long long wait_ns;                      // limit of each wait (WaitCfg)
    int expire_m;                                    // test hook: matrix whose first update wait runs out
    CUtensorMap tmw[2];                              // the work matrices of job q as [matrix][row][column]
};

__device__ __forceinline__ void gt_argmax_merge(float &v, int &i, float v2, int i2)
{
    if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
}

__device__ __forceinline__ void gt_block_argmax(float &bv, int &bi, float *red_v, int *red_i, int lane, int wid)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float v2 = __shfl_down_sync(0xffffffffu, bv, o);
        const int i2 = __shfl_down_sync(0xffffffffu, bi, o);
        gt_argmax_merge(bv, bi, v2, i2);
    }
    if (lane == 0) { red_v[wid] = bv; red_i[wid] = bi; }
}

__global__ void __launch_bounds__(kGtThreads) k_gt_init(GtJobs js)
{
    const GjJob &J = js.j[blockIdx.y];
    const int m = blockIdx.x;
    if (m >= J.count) return;
    const int n = J.n;
    const GtLayout L = gt_layout(n);
    unsigned char *sc = js.scr[blockIdx.y] + (size_t)m * L.per;
    const double *__restrict__ X = J.X + (size_t)m * J.x_stride;
    float2 *__restrict__ Wk = reinterpret_cast<float2 *>(sc + L.w);
    const int ld = gt_ld(n);
    short *used = reinterpret_cast<short *>(sc + L.used);
    unsigned char *piv = sc + L.piv;
    GtState *st = reinterpret_cast<GtState *>(sc + L.state);
    __shared__ float red_f[kGtWarps];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    float rmax = 0.f;
    for (int i = wid; i < n; i += kGtWarps) {
        float rs = 0.f;
        for (int c = lane; c < n; c += 32) {
            const double x = X[(size_t)i * n + c];
            const float h = (float)x;
            Wk[(size_t)i * ld + c] = make_float2(h, (float)(x - (double)h));
            rs += fabsf(h);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
        rmax = fmaxf(rmax, rs);
    }
    if (lane == 0) red_f[wid] = rmax;
    for (int i = t; i < n; i += kGtThreads) {
        used[i] = 0;
        piv[i] = 0;
    }
    __syncthreads();
    if (t == 0) {
        float xm = 0.f;
        for (int q = 0; q < kGtWarps; ++q) xm = fmaxf(xm, red_f[q]);
        GtState s0;
        s0.mag_h = 1.f; s0.mag_l = 0.f; s0.mag_e = 0; s0.neg = 0; s0.sing = 0; s0.xnorm = xm;
        s0.pad[0] = s0.pad[1] = 0;
        *st = s0;
    }
}

// Operand B of the update: the pivot rows before the update (zero in the panel's columns
// and for c >= w), scaled per column; one thread per column, its 32 values loaded at once.
__device__ __forceinline__ void gt_operand_b(unsigned char *sc, const GtLayout &L, int n, int jb, int w,
                                             const short *ppS)
{
    const float2 *__restrict__ Wk = reinterpret_cast<const float2 *>(sc + L.w);
    const int ld = gt_ld(n);
    int *Fcol = reinterpret_cast<int *>(sc + L.f);
    unsigned char *Bpl = sc + L.b;
    for (int col = threadIdx.x; col < n; col += blockDim.x) {
        const bool vcol = !(col >= jb && col < jb + w);
        float2 u[kGtB];
        float mx = 0.f;
#pragma unroll
        for (int c = 0; c < kGtB; ++c) {
            u[c] = (vcol && c < w) ? Wk[(size_t)ppS[c] * ld + col] : make_float2(0.f, 0.f);
            mx = fmaxf(mx, fabsf(u[c].x));
        }
        const int F = exp_bound(mx);
        Fcol[col] = F;
        const int cl = col % kGtN;
        unsigned char *base = Bpl + (size_t)(col / kGtN) * kGtSl * kGtBPlane + (cl & 7) * 2;
#pragma unroll
        for (int c = 0; c < kGtB; ++c) {
            float s7[kGtSl];
            slice_n<kGtSl>(u[c], F, s7);
            unsigned char *b = base + b_off32c(c, cl & ~7);
#pragma unroll
            for (int j = 0; j < kGtSl; ++j)
                *reinterpret_cast<__nv_bfloat16 *>(b + (size_t)j * kGtBPlane) = __float2bfloat16_rn(s7[j]);
        }
    }
}

__global__ void __launch_bounds__(kGpThreads, 1) k_gt_panel(GtJobs js)
{
    const GjJob &J = js.j[blockIdx.y];
    const int m = blockIdx.x;
    const int n = J.n, jb = js.jb;
    if (m >= J.count || jb >= n) return;
    const GtLayout L = gt_layout(n);
    unsigned char *sc = js.scr[blockIdx.y] + (size_t)m * L.per;
    GtState *st = reinterpret_cast<GtState *>(sc + L.state);
    if (st->sing) return;
    float2 *__restrict__ Wk = reinterpret_cast<float2 *>(sc + L.w);
    const int ld = gt_ld(n);
    short *pp_g = reinterpret_cast<short *>(sc + L.pp);
    short *used_g = reinterpret_cast<short *>(sc + L.used);
    unsigned char *piv_g = sc + L.piv;
    int *Erow = reinterpret_cast<int *>(sc + L.e);
    unsigned char *Apl = sc + L.a;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *P = reinterpret_cast<float2 *>(smem_raw);           // [n][32]
    short *used = reinterpret_cast<short *>(P + (size_t)n * kGtB);
    __shared__ short ppS[kGtB];
    __shared__ int red_i[kGpWarps];
    __shared__ float red_f[kGpWarps];

    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int w = min(kGtB, n - jb);
    // the previous panel's pivots stop being pivots of the current panel
    if (jb > 0 && t < kGtB) piv_g[pp_g[jb - kGtB + t]] = 0;
    for (int i = t; i < n; i += kGpThreads) used[i] = used_g[i];
    // the panel: one row of 32 per warp and step, four rows' loads in flight
    for (int i0 = wid; i0 < n; i0 += 4 * kGpWarps) {
        float2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * kGpWarps;
            v[u] = (i < n && lane < w) ? Wk[(size_t)i * ld + jb + lane] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * kGpWarps;
            if (i < n) P[i * kGtB + lane] = v[u];
        }
    }
    GtState S = *st;
    bool sing = false;
    __syncthreads();
    float bv = -1.f;
    int bi = n;
    for (int i = t; i < n; i += kGpThreads)
        if (!used[i]) gt_argmax_merge(bv, bi, fabsf(P[i * kGtB].x), i);
    gt_block_argmax(bv, bi, red_f, red_i, lane, wid);
    __syncthreads();

    // one warp per row, lane = panel column: contiguous shared-memory accesses
    const int cc = lane;
    for (int c = 0; c < w; ++c) {
        float v = red_f[0];
        int p = red_i[0];
        for (int q = 1; q < kGpWarps; ++q) gt_argmax_merge(v, p, red_f[q], red_i[q]);
        if (!(v > 0.f)) {   // every thread sees the same candidates: all leave together
            sing = true;
            break;
        }
        const float2 pv = P[p * kGtB + c];
        const float2 pinv = ff::inv(pv);
        const float2 prow = (cc == c) ? pinv : ff::mul(P[p * kGtB + cc], pinv);
        {
            const float2 a = pv.x < 0.f ? ff::neg(pv) : pv;
            const float2 mg = ff::mul(make_float2(S.mag_h, S.mag_l), a);
            int ex;
            frexpf(mg.x, &ex);
            S.mag_h = ldexpf(mg.x, -ex);
            S.mag_l = ldexpf(mg.y, -ex);
            S.mag_e += ex;
            S.neg ^= pv.x < 0.f;
        }
        if (t == 0) {
            used[p] = 1;
            ppS[c] = (short)p;
        }
        __syncthreads();                                  // the candidates and row p have been read
        if (t < kGtB) P[p * kGtB + t] = prow;
        float nbv = -1.f;
        int nbi = n;
        const int cn = c + 1;
        // four rows per step (independent chains in flight)
        constexpr int RU = 4;
        for (int i0 = wid; i0 < n; i0 += RU * kGpWarps) {
            float2 mf[RU], a[RU];
            bool live[RU];
#pragma unroll
            for (int u = 0; u < RU; ++u) {
                const int i = i0 + u * kGpWarps;
                live[u] = i < n && i != p;
                mf[u] = live[u] ? ff::neg(P[i * kGtB + c]) : make_float2(0.f, 0.f);
                // lane c: 0 + m * pinv (its prow is pinv), the same expression as the other lanes
                a[u] = (live[u] && cc != c) ? P[i * kGtB + cc] : make_float2(0.f, 0.f);
            }
            __syncwarp();                                 // every lane has read the rows' column c
#pragma unroll
            for (int u = 0; u < RU; ++u) {
                const int i = i0 + u * kGpWarps;
                if (!live[u]) continue;
                const float2 x = ff::fma2(a[u], mf[u], prow);
                P[i * kGtB + cc] = x;
                if (cc == cn && cn < w && !used[i]) gt_argmax_merge(nbv, nbi, fabsf(x.x), i);
            }
        }
        gt_block_argmax(nbv, nbi, red_f, red_i, lane, wid);
        __syncthreads();
    }
    if (sing) {
        if (t == 0) st->sing = 1;
        return;
    }
    // the eliminated panel is part of the result; bookkeeping of the pivots
    for (int i = wid; i < n; i += kGpWarps)
        if (lane < w) Wk[(size_t)i * ld + jb + lane] = P[i * kGtB + lane];
    if (t < w) {
        const int p = ppS[t];
        pp_g[jb + t] = (short)p;
        used_g[p] = 1;
        piv_g[p] = 1;
    }
    if (t == 0) {
        GtState o = *st;
        o.mag_h = S.mag_h; o.mag_l = S.mag_l; o.mag_e = S.mag_e; o.neg = S.neg;
        *st = o;
    }

    // operand A: the panel's rows, scaled per row, six slices, [row tile][slice] planes
    for (int i = wid; i < n; i += kGpWarps) {
        const float2 x = P[i * kGtB + lane];
        float mx = fabsf(x.x);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const int E = exp_bound(mx);
        float s7[kGtSl];
        slice_n<kGtSl>(x, E, s7);
        unsigned char *base = Apl + (size_t)(i >> 7) * kGtSl * kGtAPlane + a_off64(i & 127, lane >> 3) +
                              (lane & 7) * 2;
#pragma unroll
        for (int j = 0; j < kGtSl; ++j)
            *reinterpret_cast<__nv_bfloat16 *>(base + (size_t)j * kGtAPlane) = __float2bfloat16_rn(s7[j]);
        if (lane == 0) Erow[i] = E;
    }
    gt_operand_b(sc, L, n, jb, w, ppS);
}

// The panel kernel with one thread per row (n <= kGpRowMax): thread i owns row i of the
// n x 32 panel (shared memory, rows padded to 33 float pairs: conflict-free).  The 32 columns
// are eliminated in four sub-panels of 8, whose columns sit in the thread's registers: each
// pivot step updates only those 8 columns (the pivot column becomes the column of the step's
// Gauss-Jordan transformation, as in k_gt_panel); after the sub-panel its composed
// transformation T = I + W S (W: the 8 transformation columns, S: the 8 pivot rows) is
// applied to the other 24 panel columns as one rank-8 float-float update,
//   X[i][j] <- [i not a pivot of the sub-panel] X[i][j] + sum_k W[i][k] X[p_k][j],
// with the pivot rows' values from before the sub-panel.  The pivot rule (largest |entry|
// among the rows not used yet, the first on ties) and the arithmetic per multiply-add are
// those of the column-by-column elimination; the sums over a sub-panel's pivots are taken in
// pivot order.  ~3x fewer instructions than k_gt_panel.
constexpr int kGpRowMax = 544;
constexpr int kGpSub = 8;
constexpr int kGpRowLd = kGtB + 1;                       // float pairs per shared-memory row

__global__ void __launch_bounds__(kGpRowMax, 1) k_gt_panel_t(GtJobs js)
{
    const GjJob &J = js.j[blockIdx.y];
    const int m = blockIdx.x;
    const int n = J.n, jb = js.jb;
    if (m >= J.count || jb >= n) return;
    const GtLayout L = gt_layout(n);
    unsigned char *sc = js.scr[blockIdx.y] + (size_t)m * L.per;
    GtState *st = reinterpret_cast<GtState *>(sc + L.state);
    if (st->sing) return;
    float2 *__restrict__ Wk = reinterpret_cast<float2 *>(sc + L.w);
    const int ld = gt_ld(n);
    short *pp_g = reinterpret_cast<short *>(sc + L.pp);
    short *used_g = reinterpret_cast<short *>(sc + L.used);
    unsigned char *piv_g = sc + L.piv;
    int *Erow = reinterpret_cast<int *>(sc + L.e);
    unsigned char *Apl = sc + L.a;

    extern __shared__ __align__(16) unsigned char gp_smem[];
    float2 *P = reinterpret_cast<float2 *>(gp_smem);     // [blockDim.x][kGpRowLd]
    __shared__ __align__(16) float2 U_s[kGpSub][kGtB];    // the sub-panel's pivot rows, before it
    __shared__ float2 prow_s[kGpSub + 1];                 // the step's pivot row on the sub-panel, scaled; 1 / pivot
    __shared__ short ppS[kGtB];
    __shared__ int red_i[kGpRowMax / 32];
    __shared__ float red_f[kGpRowMax / 32];

    const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nwarps = blockDim.x >> 5;
    const int w = min(kGtB, n - jb);
    const int i = t;                                      // this thread's row
    const bool row_ok = i < n;
    float2 *row = P + (size_t)t * kGpRowLd;
    // the previous panel's pivots stop being pivots of the current panel
    if (jb > 0 && t < kGtB) piv_g[pp_g[jb - kGtB + t]] = 0;
    if (row_ok && w == kGtB) {
        const float4 *src = reinterpret_cast<const float4 *>(Wk + (size_t)i * ld + jb);
#pragma unroll
        for (int q = 0; q < kGtB / 2; ++q) {
            const float4 v = src[q];
            row[2 * q] = make_float2(v.x, v.y);
            row[2 * q + 1] = make_float2(v.z, v.w);
        }
    } else {
        for (int j = 0; j < kGtB; ++j) row[j] = (row_ok && j < w) ? Wk[(size_t)i * ld + jb + j] : make_float2(0.f, 0.f);
    }
    bool used = !row_ok || used_g[i] != 0;
    GtState S = *st;
    bool sing = false;

    for (int sb = 0; sb < kGtB / kGpSub && sb * kGpSub < w; ++sb) {
        const int c0 = sb * kGpSub;
        float2 xs[kGpSub];                                // the sub-panel's columns of this row
#pragma unroll
        for (int q = 0; q < kGpSub; ++q) xs[q] = row[c0 + q];
        int nk = 0;                                       // pivots of this sub-panel
        bool sub_piv = false;                             // this row is one of them
#pragma unroll
        for (int cc = 0; cc < kGpSub; ++cc) {
            if (c0 + cc >= w) break;
            // block-wide argmax of |x[c]| over the rows not used yet
            float bv = used ? -1.f : fabsf(xs[cc].x);
            int bi = used ? n : i;
            gt_block_argmax(bv, bi, red_f, red_i, lane, wid);
            __syncthreads();
            // every warp merges the warps' candidates by shuffles (the same merge rule, any order)
            float v = lane < nwarps ? red_f[lane] : -1.f;
            int p = lane < nwarps ? red_i[lane] : n;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float v2 = __shfl_xor_sync(0xffffffffu, v, o);
                const int p2 = __shfl_xor_sync(0xffffffffu, p, o);
                gt_argmax_merge(v, p, v2, p2);
            }
            if (!(v > 0.f)) {                             // every thread sees the same candidates
                sing = true;
                break;
            }
            if (i == p) {                                 // publish the pivot row (all 32 columns) and,
                for (int j = 0; j < kGtB; ++j) U_s[cc][j] = row[j];   // scaled by 1 / pivot, its
#pragma unroll                                            // sub-panel part
                for (int q = 0; q < kGpSub; ++q) U_s[cc][c0 + q] = xs[q];
                const float2 pinv_o = ff::inv(xs[cc]);
#pragma unroll
                for (int q = 0; q < kGpSub; ++q) prow_s[q] = (q == cc) ? pinv_o : ff::mul(xs[q], pinv_o);
                prow_s[kGpSub] = pinv_o;
                used = true;
                sub_piv = true;
            }
            __syncthreads();
            const float2 pv = U_s[cc][c0 + cc];
            if (t == 0) {
                const float2 a = pv.x < 0.f ? ff::neg(pv) : pv;
                const float2 mg = ff::mul(make_float2(S.mag_h, S.mag_l), a);
                int ex;
                frexpf(mg.x, &ex);
                S.mag_h = ldexpf(mg.x, -ex);
                S.mag_l = ldexpf(mg.y, -ex);
                S.mag_e += ex;
                S.neg ^= pv.x < 0.f;
                ppS[c0 + cc] = (short)p;
            }
            // the step on the sub-panel's 8 columns (the same expressions as k_gt_panel)
            const float2 mf = ff::neg(xs[cc]);
#pragma unroll
            for (int q = 0; q < kGpSub; ++q) {
                const float2 prow = prow_s[q];
                if (i == p) xs[q] = prow;
                else xs[q] = ff::fma2(q == cc ? make_float2(0.f, 0.f) : xs[q], mf, prow);
            }
            ++nk;
        }
        if (sing) break;
#pragma unroll
        for (int q = 0; q < kGpSub; ++q) row[c0 + q] = xs[q];
        // the sub-panel's transformation on the other 24 columns, pivot rows from before it
        // (two columns per pass: two independent chains, U_s read 16 bytes at a time)
        for (int j = 0; j < kGtB; j += 2) {
            if (j >= c0 && j < c0 + kGpSub) continue;
            float2 a0 = sub_piv ? make_float2(0.f, 0.f) : row[j];
            float2 a1 = sub_piv ? make_float2(0.f, 0.f) : row[j + 1];
#pragma unroll
            for (int k = 0; k < kGpSub; ++k)
                if (k < nk) {
                    const float4 u = *reinterpret_cast<const float4 *>(&U_s[k][j]);
                    a0 = ff::fma2(a0, xs[k], make_float2(u.x, u.y));
                    a1 = ff::fma2(a1, xs[k], make_float2(u.z, u.w));
                }
            row[j] = a0;
            row[j + 1] = a1;
        }
        __syncthreads();                                  // U_s is rewritten by the next sub-panel
    }
    if (sing) {
        if (t == 0) st->sing = 1;
        return;
    }
    // the eliminated panel is part of the result; bookkeeping of the pivots
    if (row_ok) {
        if (w == kGtB) {
            float4 *dst = reinterpret_cast<float4 *>(Wk + (size_t)i * ld + jb);
#pragma unroll
            for (int q = 0; q < kGtB / 2; ++q)
                dst[q] = make_float4(row[2 * q].x, row[2 * q].y, row[2 * q + 1].x, row[2 * q + 1].y);
        } else {
            for (int j = 0; j < w; ++j) Wk[(size_t)i * ld + jb + j] = row[j];
        }
    }
    if (t < w) {
        const int p = ppS[t];
        pp_g[jb + t] = (short)p;
        used_g[p] = 1;
        piv_g[p] = 1;
    }
    if (t == 0) {
        GtState o = *st;
        o.mag_h = S.mag_h; o.mag_l = S.mag_l; o.mag_e = S.mag_e; o.neg = S.neg;
        *st = o;
    }
    __syncthreads();
    // operand A: the panel's rows, scaled per row, seven slices, [row tile][slice] planes
    // (a warp per row, lane = column)
    for (int r = wid; r < n; r += nwarps) {
        const float2 xr = P[(size_t)r * kGpRowLd + lane];
        float mx = fabsf(xr.x);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const int E = exp_bound(mx);
        float s7[kGtSl];
        slice_n<kGtSl>(xr, E, s7);
        unsigned char *base = Apl + (size_t)(r >> 7) * kGtSl * kGtAPlane + a_off64(r & 127, lane >> 3) +
                              (lane & 7) * 2;
#pragma unroll
        for (int j = 0; j < kGtSl; ++j)
            *reinterpret_cast<__nv_bfloat16 *>(base + (size_t)j * kGtAPlane) = __float2bfloat16_rn(s7[j]);
        if (lane == 0) Erow[r] = E;
    }
    gt_operand_b(sc, L, n, jb, w, ppS);
}

static_assert(kGtN == kGtB, "a column tile of the update is exactly one panel");

// Bounded wait of one thread with the CTA's abort flag: false on timeout (which sets the
// flag) or as soon as another role has set it.
__device__ __forceinline__ bool gt_wait1(uint32_t mbar, uint32_t parity, uint64_t limit_ns, volatile int *abort)
{
    const uint64_t t0 = globaltimer();
    while (true) {
        if (mbar_try_wait(mbar, parity)) return true;
        if (*abort) return false;
        if (globaltimer() - t0 > limit_ns) {
            *abort = 1;
            return false;
        }
    }
}

// The same for a whole warp, which stays converged: every lane polls (the phase, once
// complete, stays complete until this warp has arrived for it), the decisions are taken
// together.  A warp left diverged here (one lane polling, the others parked) made each
// following elect.sync -- the MMA warp issues every MMA through one -- cost ~300 cycles.
__device__ __forceinline__ bool gt_wait_warp(uint32_t mbar, uint32_t parity, uint64_t limit_ns, volatile int *abort,
                                             int lane)
{
    const uint64_t t0 = globaltimer();
    while (true) {
        const bool done = mbar_try_wait(mbar, parity);
        if (__all_sync(0xffffffffu, done)) return true;
        if (__any_sync(0xffffffffu, *abort != 0)) return false;
        int late = lane == 0 && globaltimer() - t0 > limit_ns;
        late = __shfl_sync(0xffffffffu, late, 0);
        if (late) {
            if (lane == 0) *abort = 1;
            return false;
        }
    }
}

// One CTA per (matrix, tile of 128 rows), one CTA per SM, four roles:
//   X warp          the tile's old float pairs in and the updated ones out by tensor TMA
//                   (two 16-column boxes of 128 rows each way, 128-byte swizzle; rows and
//                   columns outside the matrix are zero-filled on load, clipped on store),
//                   three stages
//   B warp          bulk copies of each column tile's 7 pivot-row slice planes, three stages
//   MMA warp        the row tile's 7 panel planes (one bulk copy), then per column tile the
//                   2 K16 x 28 slice-pair MMAs into the seven accumulators (7 x 32 TMEM
//                   columns) once the epilogue has read the previous tile's
//   16 epilogue     TMEM lane quadrant x 8 columns: the seven order sums, the old values
//   warps           read from and the results written back to the stage in shared memory;
//                   first, warps 0..3 move the panel planes into TMEM, where the MMAs read
//                   them (A from TMEM: per MMA only the 1 KB B slice is read from shared
//                   memory, instead of 4 KB of A + 1 KB of B, which bounded the MMAs)
// The panel's own column tile is final and skipped.  Every wait is bounded; one that runs
// out sets the CTA's abort flag and every role leaves at its next wait; the matrix goes to
// the FP64 recomputation, and the copies and MMAs in flight drain before TMEM is freed.
__global__ void __launch_bounds__(kGtUpThreads, 1) k_gt_update(const __grid_constant__ GtJobs js, int z0)
{
    extern __shared__ __align__(1024) unsigned char gt_smem[];
    unsigned char *base = gt_smem + ((1024 - (smem_u32(gt_smem) & 1023)) & 1023);
    constexpr int kBars = 2 + 2 * kGtBs + 2 * kGtXs + 2;
    __shared__ __align__(8) uint64_t bar[kBars];
    __shared__ uint32_t tmem_slot;
    __shared__ int s_abort, s_never;

    const int z = z0 + blockIdx.z;
    const int q = z % js.nj, m = z / js.nj;
    const GjJob &J = js.j[q];
    const int n = J.n, jb = js.jb;
    const int rt = blockIdx.x;
    if (m >= J.count || jb >= n || rt * 128 >= n) return;
    const int nc = (n + kGtN - 1) / kGtN;
    const int jp = jb / kGtN;                                    // the panel's own column tile
    const int ntl = nc - 1;                                      // column tiles updated
    if (ntl == 0) return;
    const GtLayout L = gt_layout(n);
    unsigned char *sc = js.scr[q] + (size_t)m * L.per;
    const GtState *st = reinterpret_cast<const GtState *>(sc + L.state);
    if (st->sing) return;
    const int r0 = rt * 128, nr = min(128, n - r0);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const uint64_t tmap = reinterpret_cast<uint64_t>(&js.tmw[q]);

    unsigned char *As = base;                                    // 7 x 8 KB
    unsigned char *Bs = As + kGtSl * kGtAPlane;                  // 3 x 7 x 2 KB
    unsigned char *Xs = Bs + kGtBs * kGtSl * kGtBPlane;          // 3 x 2 x 16 KB
    int *Fs = reinterpret_cast<int *>(Xs + kGtXs * kGtXStage);   // [nc * 32] column exponents F_j
    float *Fsc = reinterpret_cast<float *>(Fs + nc * kGtN);      // [nc * 32] 2^F_j where |F_j| <= 60, else 0
    const uint32_t b0 = smem_u32(&bar[0]);
    const uint32_t bA = b0;
    auto BF = [&](int sb) { return b0 + 8u * (uint32_t)(1 + sb); };
    auto BE = [&](int sb) { return b0 + 8u * (uint32_t)(1 + kGtBs + sb); };
    auto XF = [&](int sx) { return b0 + 8u * (uint32_t)(1 + 2 * kGtBs + sx); };
    auto XW = [&](int sx) { return b0 + 8u * (uint32_t)(1 + 2 * kGtBs + kGtXs + sx); };
    const uint32_t bTF = b0 + 8u * (uint32_t)(1 + 2 * kGtBs + 2 * kGtXs);   // accumulators complete
    const uint32_t bTE = bTF + 8u;                                         // ... and read
    const uint32_t bAT = bTF + 16u;                                        // panel slices in TMEM
    auto col_tile = [&](int i) { return i < jp ? i : i + 1; };

    const int *Fcol = reinterpret_cast<const int *>(sc + L.f);
    // a tile whose column exponents all lie in [-60, 60] takes the fast scaling in the epilogue
    __shared__ int tile_ok[1024 / kGtN];
    if (t < 1024 / kGtN) tile_ok[t] = 1;
    __syncthreads();
    for (int c = t; c < nc * kGtN; c += kGtUpThreads) {
        const int F = c < n ? Fcol[c] : 0;
        const bool in = F >= -60 && F <= 60;
        Fs[c] = F;
        Fsc[c] = in ? __int_as_float((127 + F) << 23) : 0.f;
        if (!in) tile_ok[c / kGtN] = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;"
                     :: "r"(smem_u32(&tmem_slot)) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 32) {
        mbar_init(bA, 1);
        for (int sb = 0; sb < kGtBs; ++sb) { mbar_init(BF(sb), 1); mbar_init(BE(sb), 1); }
        for (int sx = 0; sx < kGtXs; ++sx) { mbar_init(XF(sx), 1); mbar_init(XW(sx), kGtEpWarps); }
        mbar_init(bTF, 1);
        mbar_init(bTE, kGtEpWarps);
        mbar_init(bAT, 4);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
        s_never = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    int nld = 0, nst = 0, nb = 0, nmma = 0;                      // tiles loaded / stored / copied / multiplied

    if (warp == kGtEpWarps) {
        // ---- X warp: stage sx holds tile i; before tile i + 3 is loaded into it, tile i is
        // stored and the store has finished reading the stage
        if (lane == 0) {
            auto store = [&](int i) {
                const int sx = i % kGtXs, c0 = col_tile(i) * kGtN;
                const uint32_t xs = smem_u32(Xs + sx * kGtXStage);
                tma_store_3d(tmap, xs, c0, r0, m);
                tma_store_3d(tmap, xs + kGtXStage / 2, c0 + 16, r0, m);
                bulk_commit();
                nst = i + 1;
            };
            for (int i = 0; i < ntl; ++i) {
                const int sx = i % kGtXs;
                if (i >= kGtXs) {
                    if (!gt_wait1(XW(sx), ((i / kGtXs) - 1) & 1, js.wait_ns, &s_abort)) break;
                    store(i - kGtXs);
                    bulk_wait_read0();
                }
                const int c0 = col_tile(i) * kGtN;
                const uint32_t xs = smem_u32(Xs + sx * kGtXStage);
                mbar_expect_tx(XF(sx), kGtXStage);
                tma_load_3d(tmap, xs, c0, r0, m, XF(sx));
                tma_load_3d(tmap, xs + kGtXStage / 2, c0 + 16, r0, m, XF(sx));
                nld = i + 1;
            }
            if (nld == ntl)
                for (int i = max(0, ntl - kGtXs); i < ntl; ++i) {
                    if (!gt_wait1(XW(i % kGtXs), (i / kGtXs) & 1, js.wait_ns, &s_abort)) break;
                    store(i);
                }
            bulk_wait_all0();                                    // every store complete
        }
    } else if (warp == kGtEpWarps + 1) {
        // ---- B warp
        if (lane == 0)
            for (int i = 0; i < ntl; ++i) {
                const int sb = i % kGtBs;
                if (i >= kGtBs && !gt_wait1(BE(sb), ((i / kGtBs) - 1) & 1, js.wait_ns, &s_abort)) break;
                mbar_expect_tx(BF(sb), kGtSl * kGtBPlane);
                bulk_g2s(smem_u32(Bs + sb * kGtSl * kGtBPlane), sc + L.b + (size_t)col_tile(i) * kGtSl * kGtBPlane,
                         kGtSl * kGtBPlane, BF(sb));
                nb = i + 1;
            }
    } else if (warp == kGtEpWarps + 2) {
        // ---- MMA warp: warp-uniform control flow, one elected lane issues each MMA and commit
        if (lane == 0) {
            mbar_expect_tx(bA, kGtSl * kGtAPlane);
            bulk_g2s(smem_u32(As), sc + L.a + (size_t)rt * kGtSl * kGtAPlane, kGtSl * kGtAPlane, bA);
        }
        __syncwarp();
        if (gt_wait_warp(bAT, 0, js.wait_ns, &s_abort, lane)) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t idesc = umma_idesc_f16(128, kGtN, 1);
            for (int i = 0; i < ntl; ++i) {
                const int sb = i % kGtBs;
                if (!gt_wait_warp(BF(sb), (i / kGtBs) & 1, js.wait_ns, &s_abort, lane)) break;
                if (i >= 1 && !gt_wait_warp(bTE, (i - 1) & 1, js.wait_ns, &s_abort, lane)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint64_t dB = umma_desc_sw64_mn(smem_u32(Bs + sb * kGtSl * kGtBPlane), kGtBSbo, kGtBSbo);
#pragma unroll
                for (int kk = 0; kk < kGtB / 16; ++kk)
#pragma unroll
                    for (int d = 0; d < kGtSl; ++d)
#pragma unroll
                        for (int ii = 0; ii <= d; ++ii) {
                            const int j = d - ii;
                            const uint32_t at = tmem + kGtATmem + (uint32_t)((ii * 2 + kk) * 8);
                            const uint64_t bd = dB + ((j * kGtBPlane + 2 * kk * kGtBSbo) >> 4);
                            if (kk == 0 && ii == 0) umma_bf16_ts_warp<0>(tmem + d * kGtN, at, bd, idesc);
                            else umma_bf16_ts_warp<1>(tmem + d * kGtN, at, bd, idesc);
                        }
                umma_commit_warp(BE(sb));                        // the B stage may be refilled
                umma_commit_warp(bTF);                           // the accumulators may be read
                nmma = i + 1;
            }
        }
    } else {
        // ---- epilogue warps: row r of the tile (TMEM lane), columns cg * 8 .. + 7 of each column tile
        const int quad = warp & 3, cg = warp >> 2;
        const int r = quad * 32 + lane;
        const bool row_ok = r < nr;
        const int i_row = r0 + (row_ok ? r : 0);
        const int E = row_ok ? reinterpret_cast<const int *>(sc + L.e)[i_row] : 0;
        const bool is_piv = row_ok && (sc + L.piv)[i_row] != 0;
        // 2^(E + F) as two exact multiplications by 2^E and 2^F when both lie in [-60, 60]: the
        // order sums are 0 or at least 2^-56 in magnitude (multiples of the smallest unit), so
        // the product with 2^E is a normal float, and the final rounding equals scale_pow2's
        const bool E_ok = E >= -60 && E <= 60;
        const float sE = __int_as_float((127 + (E_ok ? E : 0)) << 23);
        const uint32_t tlane = (uint32_t)(quad * 32) << 16;
        const uint32_t tl = tmem + tlane + (uint32_t)(cg * 8);
        if (warp < 4) {
            // the panel planes into TMEM columns 256 + 16 ii .. + 15: this thread's row, its 32
            // K values packed in pairs (the 64-byte swizzle of the shared-memory planes undone)
            if (gt_wait_warp(bA, 0, js.wait_ns, &s_abort, lane)) {
#pragma unroll 1
                for (int ii = 0; ii < kGtSl; ++ii) {
                    uint32_t w[16];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const uint4 u = *reinterpret_cast<const uint4 *>(As + ii * kGtAPlane + a_off64(r, c));
                        w[4 * c] = u.x; w[4 * c + 1] = u.y; w[4 * c + 2] = u.z; w[4 * c + 3] = u.w;
                    }
                    tmem_st16(tmem + tlane + kGtATmem + (uint32_t)(16 * ii), w);
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(bAT);
            }
        }
        // this thread's four 16-byte chunks of a stage (128-byte swizzle: chunk ^ (row & 7))
        const uint32_t xoff = (uint32_t)((cg >> 1) * (kGtXStage / 2) + r * 128);
        const int ck0 = (cg & 1) * 4;
        // test hook: the first panel's first wait of the chosen matrix runs out
        const bool expire = m == js.expire_m && jb == 0 && rt == 0;
        for (int i = 0; i < ntl; ++i) {
            const int sx = i % kGtXs;
            bool ok;
            if (expire && i == 0) {
                int f = 0;
                if (lane == 0) {
                    f = flag_wait(&s_never, js.wait_ns);
                    if (!f) s_abort = 1;
                }
                ok = __shfl_sync(0xffffffffu, f, 0) != 0;
            } else {
                ok = gt_wait_warp(bTF, i & 1, js.wait_ns, &s_abort, lane);
            }
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint32_t v[kGtSl][8];
#pragma unroll
            for (int d = 0; d < kGtSl; ++d) tmem_ld8_async(tl + (uint32_t)(d * kGtN), v[d]);
            tmem_wait_ld(v);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(bTE);
            // the seven order sums, exact integers in their units: orders 0..3 added as float
            // pairs, orders 4..6 (below 2^-21 of the update) first in FP32 (rounding ~2^-46)
            float hs[8], ls[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                ff::two_sum(__uint_as_float(v[0][k]), __uint_as_float(v[1][k]), hs[k], ls[k]);
                float sh, se;
                ff::two_sum(hs[k], __uint_as_float(v[2][k]), sh, se);
                ls[k] = __fadd_rn(ls[k], se);
                ff::two_sum(sh, __uint_as_float(v[3][k]), hs[k], se);
                ls[k] = __fadd_rn(ls[k], se);
                const float t456 = __fadd_rn(__uint_as_float(v[4][k]),
                                             __fadd_rn(__uint_as_float(v[5][k]), __uint_as_float(v[6][k])));
                ls[k] = __fadd_rn(ls[k], t456);
            }
            if (!gt_wait_warp(XF(sx), (i / kGtXs) & 1, js.wait_ns, &s_abort, lane)) break;
            unsigned char *xs = Xs + sx * kGtXStage + xoff;
            const int ct = col_tile(i);
            const int c0 = ct * kGtN + cg * 8;
            if (E_ok && tile_ok[ct]) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    float4 *p4 = reinterpret_cast<float4 *>(xs + (((ck0 + k) ^ (r & 7)) << 4));
                    const float4 o = *p4;
                    float2 x0 = is_piv ? make_float2(0.f, 0.f) : make_float2(o.x, o.y);
                    float2 x1 = is_piv ? make_float2(0.f, 0.f) : make_float2(o.z, o.w);
                    const float f0 = Fsc[c0 + 2 * k], f1 = Fsc[c0 + 2 * k + 1];
                    x0 = ff::add(x0, make_float2(__fmul_rn(__fmul_rn(hs[2 * k], sE), f0),
                                                 __fmul_rn(__fmul_rn(ls[2 * k], sE), f0)));
                    x1 = ff::add(x1, make_float2(__fmul_rn(__fmul_rn(hs[2 * k + 1], sE), f1),
                                                 __fmul_rn(__fmul_rn(ls[2 * k + 1], sE), f1)));
                    *p4 = make_float4(x0.x, x0.y, x1.x, x1.y);
                }
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    float4 *p4 = reinterpret_cast<float4 *>(xs + (((ck0 + k) ^ (r & 7)) << 4));
                    const float4 o = *p4;
                    float2 x0 = is_piv ? make_float2(0.f, 0.f) : make_float2(o.x, o.y);
                    float2 x1 = is_piv ? make_float2(0.f, 0.f) : make_float2(o.z, o.w);
                    const int ex0 = E + Fs[c0 + 2 * k], ex1 = E + Fs[c0 + 2 * k + 1];
                    x0 = ff::add(x0, make_float2(scale_pow2(hs[2 * k], ex0), scale_pow2(ls[2 * k], ex0)));
                    x1 = ff::add(x1, make_float2(scale_pow2(hs[2 * k + 1], ex1), scale_pow2(ls[2 * k + 1], ex1)));
                    *p4 = make_float4(x0.x, x0.y, x1.x, x1.y);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // for the TMA store
            __syncwarp();
            if (lane == 0) mbar_arrive(XW(sx));
        }
    }
    __syncthreads();
    if (s_abort && t == 0 && J.redo) J.redo[m * J.redo_stride] = 1;   // recomputed in FP64
    // nothing may land in this CTA's shared memory or TMEM after it exits: the copying
    // threads wait for their last copies, the MMA thread for its last commits (in a normal
    // run all of these have completed or complete at once)
    if (s_abort && warp == kGtEpWarps && lane == 0)
        for (int i = max(0, nld - kGtXs); i < nld; ++i) mbar_wait(XF(i % kGtXs), (i / kGtXs) & 1, kDrainNs);
    if (s_abort && warp == kGtEpWarps + 1 && lane == 0)
        for (int i = max(0, nb - kGtBs); i < nb; ++i) mbar_wait(BF(i % kGtBs), (i / kGtBs) & 1, kDrainNs);
    if (warp == kGtEpWarps + 2 && lane == 0) {
        if (s_abort) mbar_wait(bA, 0, kDrainNs);
        for (int i = max(0, nmma - kGtBs); i < nmma; ++i) mbar_wait(BE(i % kGtBs), (i / kGtBs) & 1, kDrainNs);
        if (nmma > 0) mbar_wait(bTF, (nmma - 1) & 1, kDrainNs);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" :: "r"(tmem) : "memory");
    (void)nst;
}

__global__ void __launch_bounds__(kGtThreads) k_gt_final(GtJobs js, double kappa_max)
{
    const GjJob &J = js.j[blockIdx.y];
    const int m = blockIdx.x;
    if (m >= J.count) return;
    const int n = J.n;
    const GtLayout L = gt_layout(n);
    unsigned char *sc = js.scr[blockIdx.y] + (size_t)m * L.per;
    const GtState S = *reinterpret_cast<const GtState *>(sc + L.state);
    if (S.sing) {                                        // a zero pivot in the float pairs: FP64 decides
        if (threadIdx.x == 0 && J.redo) J.redo[m * J.redo_stride] = 1;
        return;
    }
    const float2 *__restrict__ Wk = reinterpret_cast<const float2 *>(sc + L.w);
    const int ld = gt_ld(n);
    double *__restrict__ Dout = J.Dinv + (size_t)m * J.d_stride;
    const short *pp_g = reinterpret_cast<const short *>(sc + L.pp);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *tile = reinterpret_cast<float2 *>(smem_raw);        // [32][33]
    short *pp = reinterpret_cast<short *>(tile + 32 * 33);
    short *seen = pp + n;
    __shared__ float red_f[kGtWarps];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    for (int i = t; i < n; i += kGtThreads) {
        pp[i] = pp_g[i];
        seen[i] = 0;
    }
    // ||X^-1||_inf: the rows of X^-1 are the rows of the result (columns permuted)
    float imax = 0.f;
    for (int i = wid; i < n; i += kGtWarps) {
        float rs = 0.f;
        for (int c = lane; c < n; c += 32) rs += fabsf(Wk[(size_t)i * ld + c].x);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
        imax = fmaxf(imax, rs);
    }
    if (lane == 0) red_f[wid] = imax;
    __syncthreads();
    for (int kb = 0; kb < n; kb += 32) {
        for (int cb = 0; cb < n; cb += 32) {
            for (int r = wid; r < 32; r += kGtWarps) {
                const int k = kb + r, c = cb + lane;
                tile[r * 33 + lane] = (k < n && c < n) ? Wk[(size_t)pp[k] * ld + c] : make_float2(0.f, 0.f);
            }
            __syncthreads();
            for (int r = wid; r < 32; r += kGtWarps) {
                const int c = cb + r, k = kb + lane;
                if (c < n && k < n) Dout[(size_t)pp[c] * n + k] = ff::val(tile[lane * 33 + r]);
            }
            __syncthreads();
        }
    }
    if (t == 0) {
        float im = 0.f;
        for (int q = 0; q < kGtWarps; ++q) im = fmaxf(im, red_f[q]);
        const double kappa = (double)S.xnorm * (double)im;
        int par = 0;
        for (int i = 0; i < n; ++i) {
            if (seen[i]) continue;
            int len = 0, j = i;
            while (!seen[j]) { seen[j] = 1; j = pp[j]; ++len; }
            par ^= ((len & 1) == 0);
        }
        const double logabs = log((double)S.mag_h + (double)S.mag_l) + S.mag_e * 0.69314718055994530942;
        if (J.logabs) J.logabs[(size_t)m * J.la_stride] = logabs;
        if (J.sign) J.sign[(size_t)m * J.la_stride] = (par ^ S.neg) ? -1.0 : 1.0;
        if (J.redo && !(kappa <= kappa_max && isfinite(logabs))) J.redo[m * J.redo_stride] = 1;
    }
}

bool gjtc_fits(int nmax)
{
    const size_t sm = sizeof(float2) * (size_t)nmax * kGtB + sizeof(short) * (size_t)nmax;
    return nmax <= 1024 && sm + 1024 <= 227 * 1024;
}

size_t gjtc_bytes(int n_up, int n_dn, int nw)
{
    size_t b = 0;
    if (n_up > 0) b += gt_layout(n_up).per * (size_t)nw;
    if (n_dn > 0) b += gt_layout(n_dn).per * (size_t)nw;
    return b + 256;
}

// The update kernel's tensor maps: job q's work matrices as a 3-D tensor of 8-byte float
// pairs [count][n][n] (row stride gt_ld(n), matrix stride the scratch per matrix), boxes of
// 16 columns x 128 rows with 128-byte swizzle.
static cudaError_t gt_tensor_maps(GtJobs &js)
{
    for (int q = 0; q < 2; ++q) {
        memset(&js.tmw[q], 0, sizeof(CUtensorMap));
        if (q >= js.nj || js.j[q].count == 0) continue;
        const int n = js.j[q].n;
        const GtLayout L = gt_layout(n);
        const uint64_t dim[3] = {(uint64_t)n, (uint64_t)n, (uint64_t)js.j[q].count};
        const uint64_t stride[2] = {(uint64_t)gt_ld(n) * 8, (uint64_t)L.per};
        const uint32_t box[3] = {16, 128, 1};
        const cudaError_t e = tmap_encode(&js.tmw[q], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, js.scr[q] + L.w, dim,
                                          stride, box, CU_TENSOR_MAP_SWIZZLE_128B);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_gj_tc(const GjJob *jobs, int n_jobs, void *scratch, cudaStream_t st, double kappa_max,
                         const WaitCfg &wc)
{
    GtJobs js;
    int nmax = 0, cmax = 0;
    unsigned char *p = static_cast<unsigned char *>(scratch);
    for (int q = 0; q < 2; ++q) {
        js.j[q] = jobs[q < n_jobs ? q : 0];
        if (q >= n_jobs) js.j[q].count = 0;
        js.scr[q] = p;
        if (q < n_jobs) p += gt_layout(js.j[q].n).per * (size_t)js.j[q].count;
        nmax = max(nmax, js.j[q].n);
        cmax = max(cmax, js.j[q].count);
    }
    js.nj = n_jobs;
    js.jb = 0;
    js.wait_ns = wc.limit_ns;
    js.expire_m = (wc.expire_kernels & QMC_EXPIRE_A4) ? wc.expire_w : -1;
    if (cmax == 0 || n_jobs == 0) return cudaSuccess;
    if (!gjtc_fits(nmax)) return cudaErrorInvalidConfiguration;
    const size_t sm_panel = sizeof(float2) * (size_t)nmax * kGtB + sizeof(short) * (size_t)nmax;
    // 56 KB of panel slices, 3 x 14 KB of pivot-row slices, 3 x 32 KB of old values, the
    // column exponents: one CTA per SM
    const size_t sm_up = 1024 + kGtSl * (size_t)(kGtAPlane + kGtBs * kGtBPlane) + kGtXs * (size_t)kGtXStage +
                         8 * (size_t)((nmax + kGtN - 1) / kGtN * kGtN);
    const size_t sm_fin = sizeof(float2) * 32 * 33 + sizeof(short) * 2 * (size_t)nmax;
    cudaError_t e;
    if ((e = gt_tensor_maps(js)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_gt_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_panel)) !=
        cudaSuccess)
        return e;
    const int nthr_t = (nmax + 31) / 32 * 32;
    const size_t sm_t = sizeof(float2) * (size_t)nthr_t * kGpRowLd;
    if (nmax <= kGpRowMax &&
        (e = cudaFuncSetAttribute(k_gt_panel_t, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_t)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_gt_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_up)) !=
        cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_gt_final, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_fin)) !=
        cudaSuccess)
        return e;
    const dim3 g1(cmax, n_jobs);
    k_gt_init<<<g1, kGtThreads, 0, st>>>(js);
    const int nt = (nmax + 127) / 128;
    const int nz = cmax * n_jobs;
    for (int jb = 0; jb < nmax; jb += kGtB) {
        js.jb = jb;
        // one thread per row where the rows fit one CTA, else the panel in shared memory
        if (nmax <= kGpRowMax) k_gt_panel_t<<<g1, nthr_t, sm_t, st>>>(js);
        else k_gt_panel<<<g1, kGpThreads, sm_panel, st>>>(js);
        for (int z0 = 0; z0 < nz; z0 += 65535) {
            const int zn = nz - z0 < 65535 ? nz - z0 : 65535;
            k_gt_update<<<dim3(nt, 1, zn), kGtUpThreads, sm_up, st>>>(js, z0);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_gt_final<<<g1, kGtThreads, sm_fin, st>>>(js, kappa_max);
    return cudaGetLastError();
}

}  // namespace qmc
