// Step a4 of the mixed path with the panel updates on the tcgen05 tensor
// cores (a4 arithmetic QMC_A4_TENSOR).
//
// The Gauss-Jordan elimination with partial pivoting of k_gj / k_gj_ff
// (implicit pivoting: rows never move, a row map records the pivots; after
// the last panel the array holds Res with X^-1[a][b] = Res[pp[a]][ipp[b]]),
// on a float-pair work matrix (~48-bit significand), in panels of kGtB = 32
// columns, as launches over all matrices of a walker chunk:
//
//   k_gt_init    float-pair copy of X and ||X||_inf
//   per panel jb:
//   k_gt_panel   one CTA per matrix eliminates the n x 32 panel in shared
//                memory (pivot = the first row with the largest |entry| among
//                the rows not used yet: the pivots of LU with partial
//                pivoting) and writes the operands of the panel's update in
//                exact BF16 slices: the panel P [n][32] (row i scaled by
//                2^-E_i) and the pivot rows U [32][n] as they were before the
//                update (column j scaled by 2^-F_j), seven slices of 7 bits
//                each (the scheme of the C1/C5 products, one slice more)
//   k_gt_update  X[i][j] <- [i is not a pivot row of the panel] X[i][j]
//                           + sum_c P[i][c] U[c][j]
//                for every column j outside the panel; one CTA per 128 rows
//                (two CTAs per SM) loops over the 32-column tiles and issues,
//                per tile, 2 K16
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
constexpr int kGtUpThreads = 256;                    // update kernel: 4 lane quadrants x 2 column groups
constexpr int kGtN = 32;                             // columns per update tile (two CTAs per SM: 7 x 32 TMEM columns each)
constexpr int kGtSl = 7;                             // slices per operand
constexpr int kGtAcc = kGtSl;                        // one TMEM accumulator per order 0..6
constexpr uint32_t kGtAPlane = 128 * kGtB * 2;       // [128 rows][32 K] BF16, K-major, 64-byte swizzle: 8 KB
constexpr uint32_t kGtBPlane = kGtB * kGtN * 2;      // [32 K][32 columns] BF16, MN-major, 64-byte swizzle: 2 KB
constexpr uint32_t kGtBSbo = 512;                    // next group of 8 K rows (one 32-column atom each)

// MN-major, 64-byte swizzle, one 32-column atom per group of 8 K rows: byte
// offset of the 16-byte chunk holding columns n0..n0+7 of K row r
__device__ __forceinline__ uint32_t b_off32c(int r, int n0)
{
    return (uint32_t)((r >> 3) * kGtBSbo + (r & 7) * 64 + ((((n0 & 31) >> 3) ^ ((r & 7) >> 1)) << 4));
}

// tcgen05 shared-memory descriptor, 64-byte swizzle, both strides given (MN-major operand)
__device__ __forceinline__ uint64_t umma_desc_sw64_mn(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;    // SWIZZLE_64B
    return d;
}

struct GtState {                                     // per matrix, kept across the panel launches
    float mag_h, mag_l;                              // |det| = (mag_h + mag_l) 2^mag_e
    int mag_e, neg, sing;
    float xnorm;                                     // ||X||_inf
    int pad[2];
};

struct GtLayout {                                    // scratch of one matrix
    size_t a, b, e, f, pp, used, piv, state, per;
};

__host__ __device__ inline size_t gt_al(size_t x) { return (x + 255) & ~(size_t)255; }

__host__ __device__ inline GtLayout gt_layout(int n)
{
    const size_t nt = (size_t)(n + 127) / 128, nc = (size_t)(n + kGtN - 1) / kGtN;
    GtLayout L;
    size_t o = 0;
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
    float2 *__restrict__ Wk = J.work + (size_t)m * J.x_stride;
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
            Wk[(size_t)i * n + c] = make_float2(h, (float)(x - (double)h));
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
    float2 *__restrict__ Wk = J.work + (size_t)m * J.x_stride;
    short *pp_g = reinterpret_cast<short *>(sc + L.pp);
    short *used_g = reinterpret_cast<short *>(sc + L.used);
    unsigned char *piv_g = sc + L.piv;
    int *Erow = reinterpret_cast<int *>(sc + L.e);
    int *Fcol = reinterpret_cast<int *>(sc + L.f);
    unsigned char *Apl = sc + L.a, *Bpl = sc + L.b;

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
            v[u] = (i < n && lane < w) ? Wk[(size_t)i * n + jb + lane] : make_float2(0.f, 0.f);
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
        if (lane < w) Wk[(size_t)i * n + jb + lane] = P[i * kGtB + lane];
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
    // operand B: the pivot rows before the update (zero in the panel's columns and
    // for c >= w), scaled per column; one thread per column, its 32 values loaded at once
    for (int col = t; col < n; col += kGpThreads) {
        const bool vcol = !(col >= jb && col < jb + w);
        float2 u[kGtB];
        float mx = 0.f;
#pragma unroll
        for (int c = 0; c < kGtB; ++c) {
            u[c] = (vcol && c < w) ? Wk[(size_t)ppS[c] * n + col] : make_float2(0.f, 0.f);
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

// One CTA per (matrix, tile of 128 rows): the row tile's 7 A planes stay in
// shared memory; the column tiles' B planes stream through two buffers.  Per
// column tile: MMAs into the seven accumulators; once they complete, the
// accumulators are read into registers (summed as float pairs), TMEM is
// released to the next tile's MMAs, and the float-pair read-modify-write of
// the tile's rows runs while those MMAs execute.  256 threads: TMEM lane
// quadrant x two groups of 16 columns; 224 of the 256 TMEM columns and ~90 KB
// of shared memory, so that two CTAs share an SM and one's read-modify-write
// overlaps the other's.
__global__ void __launch_bounds__(kGtUpThreads, 2) k_gt_update(GtJobs js, int z0)
{
    extern __shared__ __align__(1024) unsigned char gt_smem[];
    unsigned char *base = gt_smem + ((1024 - (smem_u32(gt_smem) & 1023)) & 1023);
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_abort, s_never;

    const int z = z0 + blockIdx.z;
    const int q = z % js.nj, m = z / js.nj;
    const GjJob &J = js.j[q];
    const int n = J.n, jb = js.jb;
    const int rt = blockIdx.x;
    if (m >= J.count || jb >= n || rt * 128 >= n) return;
    const GtLayout L = gt_layout(n);
    unsigned char *sc = js.scr[q] + (size_t)m * L.per;
    const GtState *st = reinterpret_cast<const GtState *>(sc + L.state);
    if (st->sing) return;
    float2 *__restrict__ Wk = J.work + (size_t)m * J.x_stride;
    const int *Erow = reinterpret_cast<const int *>(sc + L.e);
    const int *Fcol = reinterpret_cast<const int *>(sc + L.f);
    const unsigned char *piv = sc + L.piv;
    const int w = min(kGtB, n - jb);
    const int nc = (n + kGtN - 1) / kGtN;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;

    unsigned char *As = base;                                    // 7 x 8 KB
    unsigned char *Bs0 = base + kGtSl * kGtAPlane;               // 2 x 7 x 2 KB
    int *Fs = reinterpret_cast<int *>(Bs0 + 2 * kGtSl * kGtBPlane);   // [n]
    const unsigned char *Ag = sc + L.a + (size_t)rt * kGtSl * kGtAPlane;
    auto load_b = [&](int ct) {
        const unsigned char *Bg = sc + L.b + (size_t)ct * kGtSl * kGtBPlane;
        unsigned char *Bs = Bs0 + (size_t)(ct & 1) * kGtSl * kGtBPlane;
        for (int q16 = t; q16 < (int)(kGtSl * kGtBPlane / 16); q16 += kGtUpThreads)
            cp_async16(smem_u32(Bs + 16 * q16), Bg + 16 * (size_t)q16, true);
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    for (int q16 = t; q16 < (int)(kGtSl * kGtAPlane / 16); q16 += kGtUpThreads)
        cp_async16(smem_u32(As + 16 * q16), Ag + 16 * (size_t)q16, true);
    load_b(0);                                                   // group 0: A and B(0)
    if (nc > 1) load_b(1);                                       // group 1: B(1)
    for (int c = t; c < n; c += kGtUpThreads) Fs[c] = Fcol[c];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;"
                     :: "r"(smem_u32(&tmem_slot)) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
        s_never = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t mb = smem_u32(&mbar);
    const uint32_t idesc = umma_idesc_f16(128, kGtN, 1);
    const uint32_t tlane = (uint32_t)((warp & 3) * 32) << 16;

    const int i = rt * 128 + (warp & 3) * 32 + lane;             // this thread's row (TMEM lane)
    const int cb = (warp >> 2) * 16;                             // its 16 columns of a tile
    const bool row_ok = i < n;
    const int E = row_ok ? Erow[i] : 0;
    const bool is_piv = row_ok && piv[i] != 0;
    float2 *row = Wk + (size_t)(row_ok ? i : 0) * n;
    float hs[16], ls[16];
    int ncommit = 0;

    for (int ct = 0; ct <= nc; ++ct) {
        if (ct < nc) {
            // B(ct) (and A) have landed: groups complete in order, one may stay in flight
            if (ct + 1 < nc) asm volatile("cp.async.wait_group 1;" ::: "memory");
            else asm volatile("cp.async.wait_group 0;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        __syncthreads();                                         // also: TMEM of tile ct-1 has been read
        if (s_abort) break;
        if (ct < nc && t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t dA = umma_desc_sw64(smem_u32(As), 512);
            const uint64_t dB = umma_desc_sw64_mn(smem_u32(Bs0 + (size_t)(ct & 1) * kGtSl * kGtBPlane), kGtBSbo, kGtBSbo);
#pragma unroll
            for (int kk = 0; kk < kGtB / 16; ++kk)
#pragma unroll
                for (int d = 0; d < kGtSl; ++d)
#pragma unroll
                    for (int ii = 0; ii <= d; ++ii) {
                        const int j = d - ii;
                        const uint64_t ad = dA + ((ii * kGtAPlane + 32 * kk) >> 4);
                        const uint64_t bd = dB + ((j * kGtBPlane + 2 * kk * kGtBSbo) >> 4);
                        umma_bf16(tmem + d * kGtN, ad, bd, idesc, (kk == 0 && ii == 0) ? 0u : 1u);
                    }
            umma_commit(mb);
        }
        // read-modify-write of tile ct-1 (its update is in hs/ls), overlapping the MMAs of tile ct:
        // the 16 old values are loaded first (16-byte loads where aligned), then updated and stored
        if (ct > 0 && row_ok) {
            const int c0 = (ct - 1) * kGtN + cb;
            float2 x[16];
            const bool vec = ((reinterpret_cast<uintptr_t>(row + c0) & 15) == 0) && c0 + 16 <= n;
            if (vec) {
                const float4 *r4 = reinterpret_cast<const float4 *>(row + c0);
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const float4 v4 = is_piv ? make_float4(0.f, 0.f, 0.f, 0.f) : r4[k];
                    x[2 * k] = make_float2(v4.x, v4.y);
                    x[2 * k + 1] = make_float2(v4.z, v4.w);
                }
            } else {
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    x[k] = (!is_piv && c0 + k < n) ? row[c0 + k] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int ex = E + Fs[c0 + k < n ? c0 + k : 0];
                const float2 corr = make_float2(scale_pow2(hs[k], ex), scale_pow2(ls[k], ex));
                x[k] = ff::add(x[k], corr);
            }
            const bool in_panel = c0 < jb + w && c0 + 16 > jb;   // the panel's columns are final
            if (vec && !in_panel) {
                float4 *r4 = reinterpret_cast<float4 *>(row + c0);
#pragma unroll
                for (int k = 0; k < 8; ++k) r4[k] = make_float4(x[2 * k].x, x[2 * k].y, x[2 * k + 1].x, x[2 * k + 1].y);
            } else {
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    if (c0 + k < n && !(c0 + k >= jb && c0 + k < jb + w)) row[c0 + k] = x[k];
            }
        }
        if (ct == nc) break;
        ++ncommit;
        // all leave at the next barrier; the test hook replaces the first panel's first wait of
        // the chosen matrix by one that runs out
        const bool expire = m == js.expire_m && jb == 0 && rt == 0 && ct == 0;
        if (expire ? !flag_wait(&s_never, js.wait_ns) : !mbar_wait(mb, (ncommit - 1) & 1, js.wait_ns)) s_abort = 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (ct + 2 < nc) load_b(ct + 2);                         // B buffer ct & 1 is free again
        // the seven order sums, exact integers in their units: orders 0..3 added as float
        // pairs, orders 4..6 (below 2^-21 of the update) first in FP32 (rounding ~2^-46)
        uint32_t v0[16], v1[16];
        tmem_ld16(tmem + tlane + (uint32_t)cb, v0);
        tmem_ld16(tmem + tlane + (uint32_t)(kGtN + cb), v1);
#pragma unroll
        for (int k = 0; k < 16; ++k) ff::two_sum(__uint_as_float(v0[k]), __uint_as_float(v1[k]), hs[k], ls[k]);
        tmem_ld16(tmem + tlane + (uint32_t)(2 * kGtN + cb), v0);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            float sh, se;
            ff::two_sum(hs[k], __uint_as_float(v0[k]), sh, se);
            hs[k] = sh;
            ls[k] = __fadd_rn(ls[k], se);
        }
        tmem_ld16(tmem + tlane + (uint32_t)(3 * kGtN + cb), v0);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            float sh, se;
            ff::two_sum(hs[k], __uint_as_float(v0[k]), sh, se);
            hs[k] = sh;
            ls[k] = __fadd_rn(ls[k], se);
        }
        tmem_ld16(tmem + tlane + (uint32_t)(4 * kGtN + cb), v0);
        tmem_ld16(tmem + tlane + (uint32_t)(5 * kGtN + cb), v1);
        uint32_t v2[16];
        tmem_ld16(tmem + tlane + (uint32_t)(6 * kGtN + cb), v2);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const float t456 = __fadd_rn(__uint_as_float(v0[k]),
                                         __fadd_rn(__uint_as_float(v1[k]), __uint_as_float(v2[k])));
            ls[k] = __fadd_rn(ls[k], t456);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    __syncthreads();
    if (s_abort) {                                               // recomputed in FP64
        if (t == 0 && J.redo) J.redo[m * J.redo_stride] = 1;
        asm volatile("cp.async.wait_all;" ::: "memory");
        if (ncommit > 0) mbar_wait(mb, (ncommit - 1) & 1, kDrainNs);   // let MMAs in flight drain
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" :: "r"(tmem) : "memory");
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
    const float2 *__restrict__ Wk = J.work + (size_t)m * J.x_stride;
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
        for (int c = lane; c < n; c += 32) rs += fabsf(Wk[(size_t)i * n + c].x);
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
                tile[r * 33 + lane] = (k < n && c < n) ? Wk[(size_t)pp[k] * n + c] : make_float2(0.f, 0.f);
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
    // 112 KB of operands and the column exponents; at least 120 KB so that one CTA
    // holds an SM (it allocates all 512 TMEM columns)
    // 57 KB of panel slices, 28 KB of pivot-row slices, the column exponents: two CTAs per SM
    const size_t sm_up = 1024 + kGtSl * (size_t)(kGtAPlane + 2 * kGtBPlane) + 4 * (size_t)nmax;
    const size_t sm_fin = sizeof(float2) * 32 * 33 + sizeof(short) * 2 * (size_t)nmax;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_gt_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_panel)) !=
        cudaSuccess)
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
        k_gt_panel<<<g1, kGpThreads, sm_panel, st>>>(js);
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
