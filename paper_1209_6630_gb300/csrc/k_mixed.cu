// Steps a1-a3 of the mixed-precision path.
//
// k_shell_mask   a1: per (walker, electron) bitmask of the active shells
//                (the same correctly rounded d2 < R2 decisions as the FP64 path).
// k_c15_ff       a2+a3 for C1 (the Slater matrix) and C5 (its Laplacian
//                companion): AO values and Laplacians, and the products,
//                in float-float arithmetic on the FP32 pipes (~48-bit
//                significand; the products accumulated exactly).  log|det| responds to C1 errors
//                at the 1e-10 relative level for 1000+ electrons, and the
//                kinetic energy (from C5) must hold 1e-5 of E_L even when T and
//                V nearly cancel; FP32 accumulation alone stops near 1e-6.
//                The FP32 pipe is 62x faster than the FP64 pipe on this part.
// k_tc_contract  a2+a3 for C2..C4 (the gradient matrices, i.e. the drift) on the
//                5th-generation tensor cores: tcgen05.mma kind::f16 with
//                split 16-bit operands (hi*hi + hi*lo + lo*hi) and FP32
//                accumulators in tensor memory.  FP16 splits (11 + 11
//                significant bits) with exact power-of-two scaling of both
//                operands keep each product to ~2^-22; BF16 splits (8 + 8)
//                are available for comparison (~2^-17).
//
// Tensor-core tiling.  One CTA computes, for one electron index e of one
// spin and 128 walkers (the M dimension: the same electron of different
// walkers sits near the same nucleus, so their AO lists overlap), a chunk of
// 128 MOs (N) of C2..C4.  K runs over the union of the 128 walkers' active
// AOs, 64 per step:
//   A operand (M x K, K-major, 128B swizzle): the walkers' AO gradient
//     values, computed in FP32 (four threads per walker, 16 AOs each; basis
//     tables in FP32 and positions as float pairs, so no FP64 instruction
//     runs here) and split into 16-bit hi/lo planes, zero where the walker's
//     shell is screened out;
//   B operand (N x K, MN-major, 128B swizzle): rows of the MO coefficient
//     matrix A[mu][k0..k0+127] gathered by AO index from BF16 hi/lo planes
//     prepared at system load (16-byte copies, no transpose);
//   D: three 128 x 128 FP32 accumulators (384 of the 512 TMEM columns).
// One thread issues the 36 MMAs of a K step and commits them to an mbarrier;
// waits are bounded (%globaltimer, 2 s): a wait that gives up marks the
// tile's walkers with QMC_STATUS_TIMEOUT instead of hanging.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ao_ff.cuh"
#include "ff_math.cuh"
#include "qmc_device.cuh"
#include "umma.cuh"

namespace qmc {

// ---------------------------------------------------------------- masks ----
// The decision d2 < R2 must equal the FP64 one (d2 rounded as in sqdist_rn).
// It is taken in FP32 when the FP32 value of d2 lies outside a band around R2
// that bounds its error: with S = sum_c (|r_c| + |Q_c|),
//   |d2_f32 - d2| <= 2^-20 (d2_f32 + S^2)  (input rounding 2^-24 per coordinate,
//   three roundings of the sum of squares), |R2_f32 - R2| <= 2^-24 R2;
// the band used is 2^-18 (d2_f32 + S^2 + R2_f32).  Inside the band (a few
// pairs in a thousand) the exact FP64 test decides.
constexpr int kMaskThreads = 128;

__global__ void __launch_bounds__(kMaskThreads) k_shell_mask(SysDev s, const float *__restrict__ Qf,
                                                             const float *__restrict__ aR2f,
                                                             const float *__restrict__ sR2f,
                                                             const double *__restrict__ R, int mw,
                                                             uint32_t *__restrict__ masks)
{
    extern __shared__ uint32_t mbits[];   // [mw]
    const int e = blockIdx.x, w = blockIdx.y;
    const double *r = R + ((size_t)w * s.n_elec + e) * 3;
    const double rx = r[0], ry = r[1], rz = r[2];
    const float fx = (float)rx, fy = (float)ry, fz = (float)rz;
    for (int j = threadIdx.x; j < mw; j += kMaskThreads) mbits[j] = 0u;
    __syncthreads();
    for (int a = threadIdx.x; a < s.n_atom; a += kMaskThreads) {
        const float qx = Qf[3 * a], qy = Qf[3 * a + 1], qz = Qf[3 * a + 2];
        const float dx = fx - qx, dy = fy - qy, dz = fz - qz;
        const float d2f = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
        const float S = fabsf(fx) + fabsf(qx) + fabsf(fy) + fabsf(qy) + fabsf(fz) + fabsf(qz);
        const float band0 = 0x1p-18f * (d2f + S * S);
        double d2 = -1.0;                                   // exact value, computed on demand
        auto inside = [&](float r2f, double r2) {
            const float band = band0 + 0x1p-18f * r2f;
            if (d2f < r2f - band) return true;
            if (d2f > r2f + band) return false;
            if (d2 < 0.0) d2 = sqdist_rn(rx, ry, rz, s.Q + 3 * a);
            return d2 < r2;                                 // also false for NaN
        };
        if (!inside(aR2f[a], s.atom_R2[a])) continue;
        for (int sh = s.atom_sh0[a]; sh < s.atom_sh0[a + 1]; ++sh)
            if (inside(sR2f[sh], s.sh_R2[sh])) atomicOr(&mbits[sh >> 5], 1u << (sh & 31));
    }
    __syncthreads();
    uint32_t *dst = masks + ((size_t)w * s.n_elec + e) * mw;
    for (int j = threadIdx.x; j < mw; j += kMaskThreads) dst[j] = mbits[j];
}

// Ordered list of the AOs of the shells set in `bits` (one word per thread
// slot, NT threads).  Returns the count; idx_s receives the AO indices.
template <int NT>
__device__ int aos_from_mask(const SysDev &s, const uint32_t *bits, int mw, int *idx_s, int *sh_s, int *warp_s)
{
    int words_per = (mw + NT - 1) / NT;
    const int w0 = min((int)threadIdx.x * words_per, mw), w1 = min(w0 + words_per, mw);
    int nao = 0;
    for (int j = w0; j < w1; ++j) {
        uint32_t b = bits[j];
        while (b) {
            const int bit = __ffs(b) - 1;
            b &= b - 1;
            nao += ncart(s.sh_L[j * 32 + bit]);
        }
    }
    int total;
    int off = block_excl_scan<NT>(nao, warp_s, &total);
    for (int j = w0; j < w1; ++j) {
        uint32_t b = bits[j];
        while (b) {
            const int bit = __ffs(b) - 1;
            b &= b - 1;
            const int sh = j * 32 + bit;
            const int a0 = s.sh_ao0[sh], nc = ncart(s.sh_L[sh]);
            for (int c = 0; c < nc; ++c, ++off) {
                idx_s[off] = a0 + c;
                if (sh_s) sh_s[off] = sh;
            }
        }
    }
    __syncthreads();
    return total;
}

// ------------------------------------------------ C1 and C5, FP64-accurate

// Exact float-float accumulation of a*b (a = ah + al, b = bh + bl) into a
// biased pair (sh, sl): sh starts at a power of two BIG >= 2 max|partial|, so
// |sh| >= |ah*bh| always holds and Fast2Sum is error-free; sl collects the
// rounding errors of the sums and products and the cross terms.  The value
// is (sh - BIG) + sl (the subtraction is exact).  9 FP32 instructions.
__device__ __forceinline__ void ff_acc(float ah, float al, float bh, float bl, float &sh, float &sl)
{
    const float p = __fmul_rn(ah, bh);               // _rn: never contracted into the sum below
    const float pe = fmaf(ah, bh, -p);
    const float sn = __fadd_rn(sh, p);
    const float e = __fsub_rn(p, __fsub_rn(sn, sh));
    sl = fmaf(ah, bl, sl);
    sl = fmaf(al, bh, sl);
    sl += pe + e;
    sh = sn;
}

__device__ __forceinline__ float pow2_above(float x)   // smallest power of two >= x (x > 0), 1 if x == 0
{
    if (!(x > 0.f)) return 1.f;
    int ex;
    const float m = frexpf(x, &ex);                     // x = m 2^ex, m in [0.5, 1)
    return ldexpf(1.f, m == 0.5f ? ex - 1 : ex);
}

// One CTA per (electron index e, group of G walkers).  The float-float MO
// coefficients of an AO are loaded once per thread and applied to every
// walker of the group that has the AO active (the same electron of
// neighbouring walkers sees largely the same AOs).
//
// Columns: the MO columns are split into units of 32 (one coalesced 256-byte
// load of (hi, lo) pairs per coefficient row).  With U units and W warps,
// warp w owns the q = U / W main units w, w + W, ..., and runs a loop
// compiled for q units.  The r = U - q W remaining units are shared by all
// warps along the AO list: each warp accumulates them over its 1/W slice of
// the list and the W partial sums are added in a fixed order, so every warp
// carries the same load.
//
// Union list: the CTA's AO list is the union of the G walkers' active AOs.
// It is sorted (stably, by a counting sort) by the pattern of walkers for
// which the AO is active, so each run of equal patterns is processed by a
// loop compiled for that pattern: screened-out (walker, AO) pairs cost no
// instruction.  The AO values of up to kC15Chunk union AOs are staged at
// once; a larger union is handled in several chunks whose partial sums are
// added in global memory.
constexpr int kC15Warps = 8;                       // warps when there are >= 8 units
constexpr int kC15MaxThreads = 32 * kC15Warps;
constexpr int kC15Chunk = 1024;

struct C15Args {
    SysDev s;
    FfBasis fb;
    int nw, mw;
    const double *R;
    const uint32_t *masks;
    const float2 *A[2];                            // (hi, lo) coefficient planes [n_ao][ns32]
    int ns32[2];
    const float *cmax[2];
    double *X, *L5;
};

// Accumulators of NU column units for the G walkers, and the coefficient
// pipeline (the AO being accumulated and the next one).
template <int NU, int G>
struct C15Acc {
    float vh[G][NU], vl[G][NU], lh[G][NU], ll[G][NU];
    float2 a[NU], n[NU];
};

constexpr int popc_const(int x) { return x ? (x & 1) + popc_const(x >> 1) : 0; }

// Units of a warp are kC15Warps units apart (a compile-time stride).
template <int NU, int G, int P>
__device__ __forceinline__ void c15_run(C15Acc<NU, G> &acc, int m, int m_end, int k0, const int *__restrict__ idx_s,
                                        const float4 *__restrict__ b_s, const float2 *__restrict__ A, int ns32,
                                        int col0)
{
    // unrolled so that the running sums and the prefetch ring rotate through
    // registers instead of being copied at the end of every iteration; only
    // the common patterns (all walkers, all but one) are unrolled, to keep
    // the code within the instruction cache
    constexpr int kPop = popc_const(P);
    constexpr int kUnroll = kPop == G ? 4 : (kPop == G - 1 ? 2 : 1);
#pragma unroll kUnroll
    for (; m < m_end; ++m) {
        const float2 *row = A + (size_t)idx_s[m + 2] * ns32 + col0;    // two AOs ahead (the list is padded)
        float2 f[NU];
#pragma unroll
        for (int j = 0; j < NU; ++j) f[j] = __ldg(row + 32 * kC15Warps * j);
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (((P >> g) & 1) != 0) {              // constant after unrolling
                const float4 b = b_s[g * kC15Chunk + (m - k0)];
#pragma unroll
                for (int j = 0; j < NU; ++j) {
                    ff_acc(acc.a[j].x, acc.a[j].y, b.x, b.y, acc.vh[g][j], acc.vl[g][j]);
                    ff_acc(acc.a[j].x, acc.a[j].y, b.z, b.w, acc.lh[g][j], acc.ll[g][j]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < NU; ++j) { acc.a[j] = acc.n[j]; acc.n[j] = f[j]; }
    }
}

template <int NU, int G, int P>
__device__ __forceinline__ void c15_dispatch(int p, C15Acc<NU, G> &acc, int m, int m_end, int k0,
                                             const int *idx_s, const float4 *b_s, const float2 *A, int ns32,
                                             int col0)
{
    if constexpr (P < (1 << G)) {
        if (p == P) c15_run<NU, G, P>(acc, m, m_end, k0, idx_s, b_s, A, ns32, col0);
        else c15_dispatch<NU, G, P + 1>(p, acc, m, m_end, k0, idx_s, b_s, A, ns32, col0);
    }
}

// Biased sums over the AOs [ma, mb) of the chunk starting at k0, for the
// units of columns col0 + 32 kC15Warps j (j < NU) of the lane.
template <int NU, int G>
__device__ __forceinline__ void c15_accumulate(C15Acc<NU, G> &acc, const float (&bias_v)[G][NU],
                                               const float (&bias_l)[G][NU], int ma, int mb, int k0,
                                               const int *__restrict__ idx_s, const int *__restrict__ seg_s,
                                               const float4 *__restrict__ b_s, const float2 *__restrict__ A,
                                               int ns32, int col0)
{
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
        for (int j = 0; j < NU; ++j) {
            acc.vh[g][j] = bias_v[g][j];
            acc.lh[g][j] = bias_l[g][j];
            acc.vl[g][j] = 0.f;
            acc.ll[g][j] = 0.f;
        }
    if (ma >= mb) return;
    {
        const float2 *r0 = A + (size_t)idx_s[ma] * ns32 + col0, *r1 = A + (size_t)idx_s[ma + 1] * ns32 + col0;
#pragma unroll
        for (int j = 0; j < NU; ++j) {
            acc.a[j] = __ldg(r0 + 32 * kC15Warps * j);
            acc.n[j] = __ldg(r1 + 32 * kC15Warps * j);
        }
    }
    for (int p = 1; p < (1 << G); ++p) {
        const int m = max(seg_s[p], ma), m_end = min(seg_s[p + 1], mb);
        if (m < m_end) c15_dispatch<NU, G, 1>(p, acc, m, m_end, k0, idx_s, b_s, A, ns32, col0);
    }
}

__device__ __forceinline__ size_t c15_row_offset(const SysDev &s, int w, int spin, int ei, int ns)
{
    const size_t msz = (size_t)s.n_up * s.n_up + (size_t)s.n_dn * s.n_dn;
    return (size_t)w * msz + (spin ? (size_t)s.n_up * s.n_up : 0) + (size_t)ei * ns;
}

// The NU main units of a warp (unit w + kC15Warps j): accumulate over the
// whole chunk and add to the outputs.
template <int NU, int G>
__device__ __forceinline__ void c15_main(const C15Args &a, int spin, int ei, int ns, int w0, int ng, int k0, int kc,
                                         const int *idx_s, const int *seg_s, const float4 *b_s,
                                         const float (*bsum_s)[2])
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const float2 *__restrict__ A = spin ? a.A[1] : a.A[0];
    const float *__restrict__ cmax = spin ? a.cmax[1] : a.cmax[0];
    const int ns32 = spin ? a.ns32[1] : a.ns32[0];
    const int col0 = wid * 32 + lane;
    float bias_v[G][NU], bias_l[G][NU];
#pragma unroll
    for (int j = 0; j < NU; ++j) {
        const float cm = cmax[col0 + 32 * kC15Warps * j];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            bias_v[g][j] = pow2_above(2.f * cm * bsum_s[g][0]);
            bias_l[g][j] = pow2_above(2.f * cm * bsum_s[g][1]);
        }
    }
    C15Acc<NU, G> acc;
    c15_accumulate<NU, G>(acc, bias_v, bias_l, k0, k0 + kc, k0, idx_s, seg_s, b_s, A, ns32, col0);
    // (sh - BIG) is exact; add the chunk's sums to the outputs
#pragma unroll
    for (int g = 0; g < G; ++g) {
        if (g >= ng) break;
        const size_t off = c15_row_offset(a.s, w0 + g, spin, ei, ns);
#pragma unroll
        for (int j = 0; j < NU; ++j) {
            const int k = col0 + 32 * kC15Warps * j;
            if (k >= ns) continue;
            const double v = (double)(acc.vh[g][j] - bias_v[g][j]) + (double)acc.vl[g][j];
            const double lp = (double)(acc.lh[g][j] - bias_l[g][j]) + (double)acc.ll[g][j];
            if (k0 == 0) { a.X[off + k] = v; a.L5[off + k] = lp; }
            else { a.X[off + k] += v; a.L5[off + k] += lp; }
        }
    }
}

// One remainder unit: this warp's partial sums over its slice of the chunk,
// written to part_s[wid][g][o][lane].
template <int G>
__device__ __forceinline__ void c15_slice(const C15Args &a, int spin, int unit, int nwarps, int k0, int kc,
                                          const int *idx_s, const int *seg_s, const float4 *b_s,
                                          const float (*bsum_s)[2], double *part_s)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const float2 *__restrict__ A = spin ? a.A[1] : a.A[0];
    const float *__restrict__ cmax = spin ? a.cmax[1] : a.cmax[0];
    const int ns32 = spin ? a.ns32[1] : a.ns32[0];
    const int col0 = unit * 32 + lane;
    const int ma = k0 + (int)((long long)kc * wid / nwarps), mb = k0 + (int)((long long)kc * (wid + 1) / nwarps);
    float bias_v[G][1], bias_l[G][1];
    const float cm = cmax[col0];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        bias_v[g][0] = pow2_above(2.f * cm * bsum_s[g][0]);
        bias_l[g][0] = pow2_above(2.f * cm * bsum_s[g][1]);
    }
    C15Acc<1, G> acc;
    c15_accumulate<1, G>(acc, bias_v, bias_l, ma, mb, k0, idx_s, seg_s, b_s, A, ns32, col0);
#pragma unroll
    for (int g = 0; g < G; ++g) {
        part_s[((wid * G + g) * 2 + 0) * 32 + lane] = (double)(acc.vh[g][0] - bias_v[g][0]) + (double)acc.vl[g][0];
        part_s[((wid * G + g) * 2 + 1) * 32 + lane] = (double)(acc.lh[g][0] - bias_l[g][0]) + (double)acc.ll[g][0];
    }
}

template <int NQ, int G>
__global__ void __launch_bounds__(kC15MaxThreads, 2) k_c15_ff(C15Args a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *b_s = reinterpret_cast<float4 *>(smem_raw);            // [G][kC15Chunk]: (vh, vl, lh, ll)
    double *part_s = reinterpret_cast<double *>(b_s + G * kC15Chunk);   // [warps][G][2][32] remainder partials
    uint32_t *mk_s = reinterpret_cast<uint32_t *>(part_s + kC15Warps * G * 64);   // [G][mw]
    uint32_t *un_s = mk_s + G * a.mw;                               // [mw]
    int *idx_s = reinterpret_cast<int *>(un_s + a.mw);              // [n_ao + 2], sorted union list
    int *tmp_s = reinterpret_cast<int *>(b_s);                      // unsorted list (b_s is free then)
    __shared__ int warp_s[kC15Warps];
    __shared__ float bsum_s[G][2];                                  // sum |b| per walker and output
    __shared__ float2 r_s[G][3];                                    // walker positions as float pairs
    __shared__ int seg_s[(1 << G) + 1];                             // start of each pattern's run

    const SysDev &s = a.s;
    const int mw = a.mw;
    const int e = blockIdx.x, t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int nthr = blockDim.x, nwarps = nthr >> 5;
    const int w0 = blockIdx.y * G;
    const int ng = min(G, a.nw - w0);
    const int spin = e >= s.n_up;
    const int ei = spin ? e - s.n_up : e;
    const int ns = spin ? s.n_dn : s.n_up;

    for (int q = t; q < G * mw; q += nthr) {
        const int g = q / mw, j = q - g * mw;
        mk_s[q] = (g < ng) ? a.masks[((size_t)(w0 + g) * s.n_elec + e) * mw + j] : 0u;
    }
    if (t < 3 * G) {
        const int g = t / 3, c = t - 3 * g;
        r_s[g][c] = (g < ng) ? ff::from_double(a.R[((size_t)(w0 + g) * s.n_elec + e) * 3 + c]) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int j = t; j < mw; j += nthr) {
        uint32_t u = 0;
#pragma unroll
        for (int g = 0; g < G; ++g) u |= mk_s[g * mw + j];
        un_s[j] = u;
    }
    __syncthreads();
    const int K = aos_from_mask_n(s, un_s, mw, tmp_s, warp_s);

    // activity pattern of every union AO, packed above the AO index
    for (int m = t; m < K; m += nthr) {
        const int mu = tmp_s[m], sh = s.ao_shell[mu];
        int p = 0;
#pragma unroll
        for (int g = 0; g < G; ++g) p |= (int)((mk_s[g * mw + (sh >> 5)] >> (sh & 31)) & 1u) << g;
        tmp_s[m] = mu | (p << 24);
    }
    if (t <= (1 << G)) seg_s[t] = 0;
    __syncthreads();
    // stable counting sort by pattern (one warp; deterministic order)
    if (wid == 0) {
        for (int m0 = 0; m0 < K; m0 += 32) {
            const int m = m0 + lane;
            const int p = m < K ? (tmp_s[m] >> 24) : (1 << G);
            const unsigned same = __match_any_sync(0xffffffffu, p);
            if (m < K && lane == __ffs(same) - 1) seg_s[p + 1] += __popc(same);
            __syncwarp();
        }
        if (lane == 0)
            for (int p = 1; p <= (1 << G); ++p) seg_s[p] += seg_s[p - 1];
        __syncwarp();
        // seg_s[p] holds the start of pattern p's run; place the entries
        for (int m0 = 0; m0 < K; m0 += 32) {
            const int m = m0 + lane;
            const int v = m < K ? tmp_s[m] : 0;
            const int p = m < K ? (v >> 24) : (1 << G);
            const unsigned same = __match_any_sync(0xffffffffu, p);
            int pos = 0;
            if (m < K) pos = seg_s[p] + __popc(same & ((1u << lane) - 1u));
            __syncwarp();
            if (m < K) {
                idx_s[pos] = v & 0xffffff;
                if (lane == __ffs(same) - 1) seg_s[p] += __popc(same);
            }
            __syncwarp();
        }
        // seg_s[p] is now the end of run p, i.e. the start of run p + 1
        if (lane == 0) {
            for (int p = (1 << G); p >= 1; --p) seg_s[p] = seg_s[p - 1];
            seg_s[0] = 0;
            idx_s[K] = K > 0 ? idx_s[K - 1] : 0;     // padding read by the two-ahead prefetch
            idx_s[K + 1] = idx_s[K];
        }
    }
    __syncthreads();

    // column units of this spin: q main units per warp (when a loop is
    // compiled for that count, else none) and r units shared along the list
    const int U = (ns + 31) >> 5;
    int q = U / nwarps;
    if (q != NQ && (NQ == 1 || q != NQ - 1)) q = 0;
    const int r = U - q * nwarps;

    for (int k0 = 0; k0 < K; k0 += kC15Chunk) {
        const int kc = min(kC15Chunk, K - k0);
        // float-float values and Laplacians, one (walker, AO) per thread and step
        for (int qq = t; qq < G * kc; qq += nthr) {
            const int g = qq / kc, m = qq - g * kc;
            const int mu = idx_s[k0 + m];
            const int sh = s.ao_shell[mu];
            float4 b = make_float4(0.f, 0.f, 0.f, 0.f);
            if (g < ng && ((mk_s[g * mw + (sh >> 5)] >> (sh & 31)) & 1u)) {
                float2 v, lp;
                ao_val_lap_ff(s, a.fb, mu, r_s[g], v, lp);
                b = make_float4(v.x, v.y, lp.x, lp.y);
            }
            b_s[g * kC15Chunk + m] = b;
        }
        __syncthreads();
        // sum |b_hi| per (walker, output), one warp each, fixed order (deterministic bias)
        for (int go = wid; go < 2 * G; go += nwarps) {
            const int g = go >> 1, o = go & 1;
            float acc = 0.f;
            for (int m = lane; m < kc; m += 32) {
                const float4 b = b_s[g * kC15Chunk + m];
                acc += fabsf(o ? b.z : b.x);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if (lane == 0) bsum_s[g][o] = acc;
        }
        __syncthreads();
        // main units (q is the same for every warp)
        if (q == NQ) c15_main<NQ, G>(a, spin, ei, ns, w0, ng, k0, kc, idx_s, seg_s, b_s, bsum_s);
        else if constexpr (NQ > 1) {
            if (q == NQ - 1) c15_main<NQ - 1, G>(a, spin, ei, ns, w0, ng, k0, kc, idx_s, seg_s, b_s, bsum_s);
        }
        // remainder units, split along the AO list
        for (int i = 0; i < r; ++i) {
            const int unit = q * nwarps + i;
            c15_slice<G>(a, spin, unit, nwarps, k0, kc, idx_s, seg_s, b_s, bsum_s, part_s);
            __syncthreads();
            for (int qq = t; qq < G * 64; qq += nthr) {
                const int g = qq >> 6, o = (qq >> 5) & 1, l = qq & 31;
                const int k = unit * 32 + l;
                if (g >= ng || k >= ns) continue;
                double v = 0.0;
                for (int w = 0; w < nwarps; ++w) v += part_s[((w * G + g) * 2 + o) * 32 + l];
                double *dst = (o ? a.L5 : a.X) + c15_row_offset(s, w0 + g, spin, ei, ns) + k;
                if (k0 == 0) *dst = v;
                else *dst += v;
            }
            __syncthreads();
        }
        __syncthreads();
    }
    if (K == 0) {   // no active AO for any walker of the group: zero rows
        for (int g = 0; g < ng; ++g) {
            const size_t off = c15_row_offset(s, w0 + g, spin, ei, ns);
            for (int k = t; k < ns; k += nthr) { a.X[off + k] = 0.0; a.L5[off + k] = 0.0; }
        }
    }
}

// ------------------------------------------------------------ tcgen05 path
struct TcArgs {
    SysDev s;
    const double *R;
    const uint32_t *masks;
    int mw;
    int nw;                  // walkers in this chunk
    TcTables tt;             // 16-bit hi/lo planes of A [n_ao][ns_pad] and scales
    float *Cg;               // [nw][3][msz] FP32 (C2..C4)
    uint32_t *wstatus;       // [nw] per-walker status (QMC_STATUS_TIMEOUT on a timed-out wait)
    unsigned long long wait_ns;   // limit of each wait for the MMAs
};

__global__ void __launch_bounds__(kTcThreads, 1) k_tc_contract(TcArgs p)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    // operands first (1024-aligned), then bookkeeping
    unsigned char *base = tc_smem + ((1024 - (smem_u32(tc_smem) & 1023)) & 1023);
    unsigned char *As = base;                                  // 6 planes [out l][split]
    unsigned char *Bs = base + 2 * TC_OUT * kAPlaneBytes;      // 2 planes [split]
    uint32_t *mask_s = reinterpret_cast<uint32_t *>(Bs + 2 * kBPlaneBytes);   // [128][mw]
    int *ao_s = reinterpret_cast<int *>(mask_s + TC_M * p.mw);                // [n_ao + 64]
    __shared__ uint32_t union_s[256];
    __shared__ int warp_s[kTcThreads / 32];
    __shared__ int4 meta_s[2][TC_K];                           // {mu, shell, atom, first primitive}
    __shared__ int4 meta2_s[2][TC_K];                          // {primitives, powers, scale bits, -}
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_abort;

    const SysDev &s = p.s;
    const int t = threadIdx.x, warp = t >> 5;
    const int row = t & (TC_M - 1), kq = t >> 7;      // walker row, quarter of the K step
    const int e = blockIdx.y;
    const int spin = e >= s.n_up;
    const int ei = spin ? e - s.n_up : e;
    const int ns = spin ? s.n_dn : s.n_up;
    const int k0 = blockIdx.x * TC_N;
    if (k0 >= ns) return;
    const int nspad = p.tt.ns_pad[spin];
    const int f16 = p.tt.f16;
    const int ncols = min(TC_N, nspad - k0);   // multiple of 64
    const int w = blockIdx.z * TC_M + row;     // this thread's walker
    const bool wvalid = w < p.nw;
    const int mw = p.mw;

    // masks of the tile's walkers and their union
    for (int q = t; q < TC_M * mw; q += kTcThreads) {
        const int m = q / mw, j = q - m * mw;
        const int wm = blockIdx.z * TC_M + m;
        mask_s[q] = (wm < p.nw) ? p.masks[((size_t)wm * s.n_elec + e) * mw + j] : 0u;
    }
    if (t == 0) s_abort = 0;
    __syncthreads();
    for (int j = t; j < mw; j += kTcThreads) {
        uint32_t u = 0;
        for (int m = 0; m < TC_M; ++m) u |= mask_s[m * mw + j];
        union_s[j] = u;
    }
    __syncthreads();
    const int KU = aos_from_mask<kTcThreads>(s, union_s, mw, ao_s, nullptr, warp_s);
    const int nks = (KU + TC_K - 1) / TC_K;
    for (int q = KU + t; q < nks * TC_K; q += kTcThreads) ao_s[q] = -1;

    // TMEM: 4 accumulators x 128 columns
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;"
                     :: "r"(smem_u32(&tmem_slot)) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t mbar_a = smem_u32(&mbar);
    const uint32_t idesc = umma_idesc_f16(TC_M, ncols, f16 ? 0 : 1);
    const uint64_t kWait = p.wait_ns;

    // this walker's position as float pairs (hi + lo)
    const double *rw = p.R + ((size_t)(wvalid ? w : 0) * s.n_elec + e) * 3;
    const float rxh = (float)rw[0], ryh = (float)rw[1], rzh = (float)rw[2];
    const float rxl = (float)(rw[0] - (double)rxh), ryl = (float)(rw[1] - (double)ryh),
                rzl = (float)(rw[2] - (double)rzh);
    const uint32_t *my_mask = mask_s + row * mw;
    const float *__restrict__ pgf = p.tt.pgf;
    const float *__restrict__ pcf = p.tt.pcf;
    const float *__restrict__ scf = p.tt.scf;
    const float *__restrict__ Qhi = p.tt.Qhi;
    const float *__restrict__ Qlo = p.tt.Qlo;
    const uint16_t *__restrict__ Bhi = p.tt.hi[spin];
    const uint16_t *__restrict__ Blo = p.tt.lo[spin];
    const float isc0 = p.tt.in_scale[0], isc1 = p.tt.in_scale[1], isc2 = p.tt.in_scale[2];

    // Per K step, the 64 AOs' metadata is staged in shared memory one step
    // ahead (threads 0..63 walk AO -> shell -> atom / primitives while the
    // step before is being produced); the B rows of a step are loaded into
    // registers first, and the first 8 AO gradients of a thread are computed
    // before waiting for the previous step's MMAs, which therefore overlap
    // the production.  The radial part is computed once per shell.
    auto load_meta = [&](int ks_, int4 &m0, int4 &m1) {
        const int mu = ao_s[ks_ * TC_K + t];
        if (mu >= 0) {
            const int sh = s.ao_shell[mu];
            m0 = make_int4(mu, sh, s.sh_atom[sh], s.sh_pstart[sh]);
            m1 = make_int4(s.sh_nprim[sh], s.ao_pow[mu], __float_as_int(scf[mu]), 0);
        } else {
            m0 = make_int4(-1, 0, 0, 0);
            m1 = make_int4(0, 0, 0, 0);
        }
    };
    if (t < TC_K && nks > 0) {
        int4 m0, m1;
        load_meta(0, m0, m1);
        meta_s[0][t] = m0;
        meta2_s[0][t] = m1;
    }
    __syncthreads();

    constexpr int kBChunks = 2 * TC_K * (TC_N / 8) / kTcThreads;   // 16-byte B chunks per thread
    for (int ks = 0; ks < nks; ++ks) {
        const int buf = ks & 1;
        const bool has_next = ks + 1 < nks;
        int4 nm0 = make_int4(-1, 0, 0, 0), nm1 = make_int4(0, 0, 0, 0);
        if (t < TC_K && has_next) load_meta(ks + 1, nm0, nm1);
        // B operand rows A[mu][k0 .. k0+127] of both planes, into registers
        uint4 bv[kBChunks];
#pragma unroll
        for (int j = 0; j < kBChunks; ++j) {
            const int q = t + j * kTcThreads;
            const int plane = q / (TC_K * (TC_N / 8));
            const int rem = q - plane * (TC_K * (TC_N / 8));
            const int r = rem / (TC_N / 8), c = rem - r * (TC_N / 8);
            const int mu = meta_s[buf][r].x;
            bv[j] = make_uint4(0u, 0u, 0u, 0u);
            if (mu >= 0 && 8 * c < ncols)
                bv[j] = __ldg(reinterpret_cast<const uint4 *>((plane ? Blo : Bhi) + (size_t)mu * nspad + k0 + 8 * c));
        }
        // A operand: gradient values of 16 AOs (this thread's quarter) for walker `row`, 8 at a time
        {
            int last_atom = -1, last_sh = -1;
            float dx = 0.f, dy = 0.f, dz = 0.f, d2 = 0.f, g = 0.f, gd = 0.f;
            for (int h = 0; h < 2; ++h) {
                float v[TC_OUT][8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int4 m0 = meta_s[buf][kq * 16 + 8 * h + q];
                    const int sh = m0.y;
                    float g1 = 0.f, g2 = 0.f, g3 = 0.f;
                    if (m0.x >= 0 && wvalid && ((my_mask[sh >> 5] >> (sh & 31)) & 1u)) {
                        const int4 m1 = meta2_s[buf][kq * 16 + 8 * h + q];
                        const int a = m0.z;
                        if (a != last_atom) {
                            last_atom = a;
                            dx = (rxh - Qhi[3 * a]) + (rxl - Qlo[3 * a]);
                            dy = (ryh - Qhi[3 * a + 1]) + (ryl - Qlo[3 * a + 1]);
                            dz = (rzh - Qhi[3 * a + 2]) + (rzl - Qlo[3 * a + 2]);
                            d2 = dx * dx + dy * dy + dz * dz;
                        }
                        if (sh != last_sh) {
                            last_sh = sh;
                            g = 0.f;
                            gd = 0.f;
                            for (int pr = 0; pr < m1.x; ++pr) {
                                const float gam = pgf[m0.w + pr];
                                const float ce = pcf[m0.w + pr] * expf(-gam * d2);
                                g += ce;
                                gd += gam * ce;
                            }
                        }
                        const int pw = m1.y;
                        const int nx = pw & 255, ny = (pw >> 8) & 255, nz = (pw >> 16) & 255;
                        auto ip = [](float x, int n) {
                            float y = 1.f;
                            for (int i = 0; i < n; ++i) y *= x;
                            return y;
                        };
                        const float px = ip(dx, nx), py = ip(dy, ny), pz = ip(dz, nz);
                        const float P = px * py * pz;
                        const float dpx = nx ? nx * ip(dx, nx - 1) : 0.f;
                        const float dpy = ny ? ny * ip(dy, ny - 1) : 0.f;
                        const float dpz = nz ? nz * ip(dz, nz - 1) : 0.f;
                        const float c = __int_as_float(m1.z);
                        const float m2gd = -2.f * gd;
                        g1 = c * (dpx * py * pz * g + m2gd * dx * P);
                        g2 = c * (px * dpy * pz * g + m2gd * dy * P);
                        g3 = c * (px * py * dpz * g + m2gd * dz * P);
                    }
                    v[0][q] = g1 * isc0; v[1][q] = g2 * isc1; v[2][q] = g3 * isc2;
                }
                if (h == 0) {
                    // the previous step's MMAs read the operand buffers: wait before overwriting them
                    if (ks > 0 && !mbar_wait(mbar_a, (ks - 1) & 1, kWait)) s_abort = 1;
                    __syncthreads();
                    if (s_abort) break;
                }
                const int c8 = kq * 2 + h;
#pragma unroll
                for (int l = 0; l < TC_OUT; ++l) {
                    uint32_t hi[4], lo[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) split2(v[l][2 * q], v[l][2 * q + 1], f16, hi[q], lo[q]);
                    const uint32_t off = a_off(row, c8);
                    *reinterpret_cast<uint4 *>(As + (2 * l) * kAPlaneBytes + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                    *reinterpret_cast<uint4 *>(As + (2 * l + 1) * kAPlaneBytes + off) =
                        make_uint4(lo[0], lo[1], lo[2], lo[3]);
                }
            }
        }
        if (s_abort) break;
#pragma unroll
        for (int j = 0; j < kBChunks; ++j) {
            const int q = t + j * kTcThreads;
            const int plane = q / (TC_K * (TC_N / 8));
            const int rem = q - plane * (TC_K * (TC_N / 8));
            const int r = rem / (TC_N / 8), c = rem - r * (TC_N / 8);
            *reinterpret_cast<uint4 *>(Bs + plane * kBPlaneBytes + b_off(r, 8 * c)) = bv[j];
        }
        if (t < TC_K && has_next) {
            meta_s[buf ^ 1][t] = nm0;
            meta2_s[buf ^ 1][t] = nm1;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if ((t >> 5) == 0) {                          // converged warp: elect.sync per MMA
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
#pragma unroll
            for (int kk = 0; kk < TC_K / 16; ++kk) {
                const uint64_t bh = umma_desc(b0 + 2 * kk * kBSbo, kBLbo, kBSbo);
                const uint64_t bl = umma_desc(b0 + kBPlaneBytes + 2 * kk * kBSbo, kBLbo, kBSbo);
#pragma unroll
                for (int l = 0; l < TC_OUT; ++l) {
                    const uint64_t ah = umma_desc(a0 + (2 * l) * kAPlaneBytes + 32 * kk, 16, 1024);
                    const uint64_t al = umma_desc(a0 + (2 * l + 1) * kAPlaneBytes + 32 * kk, 16, 1024);
                    const uint32_t d = tmem + l * TC_N;
                    umma_bf16_warp(d, ah, bh, idesc, (ks > 0 || kk > 0) ? 1u : 0u);
                    umma_bf16_warp(d, ah, bl, idesc, 1u);
                    umma_bf16_warp(d, al, bh, idesc, 1u);
                }
            }
            umma_commit_warp(mbar_a);
        }
    }

    bool ok = !s_abort;
    if (ok && nks > 0) ok = mbar_wait(mbar_a, (nks - 1) & 1, kWait);
    if (!ok) {
        if (wvalid) atomicOr(p.wstatus + w, (uint32_t)QMC_STATUS_TIMEOUT);
        // let any MMA still in flight drain (bounded) before freeing TMEM
        if (nks > 0) mbar_wait(mbar_a, (nks - 1) & 1, kDrainNs);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    // epilogue: TMEM -> registers -> C2..C4 rows of this walker
    const size_t msz = (size_t)s.n_up * s.n_up + (size_t)s.n_dn * s.n_dn;
    const size_t nss = (size_t)ns * ns;
    float *crow = p.Cg + (size_t)(wvalid ? w : 0) * TC_OUT * msz + (spin ? TC_OUT * (size_t)s.n_up * s.n_up : 0) +
                  (size_t)ei * ns;
    for (int l = 0; l < TC_OUT; ++l) {
        for (int cb = (warp >> 2) * 32; cb < ncols; cb += 32 * (kTcThreads / 128)) {   // warps w, w+4, ... share lanes
            uint32_t v[32];
            const uint32_t ta = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(l * TC_N + cb);
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                         "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                         "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                           "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
                           "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
                           "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
                           "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
                           "=r"(v[31])
                         : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (wvalid && ok) {
                float *dst = crow + (size_t)l * nss + k0 + cb;
                const float osc = p.tt.out_scale[spin][l];
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    if (k0 + cb + q < ns) dst[q] = (nks > 0) ? __uint_as_float(v[q]) * osc : 0.f;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" :: "r"(tmem) : "memory");
}

// --------------------------------------------------------------- launchers
cudaError_t launch_shell_mask(const SysDev &s, const MixedTables &mt, int nw, const double *R, int mw,
                              uint32_t *masks, cudaStream_t st)
{
    if (nw == 0) return cudaSuccess;
    dim3 grid(s.n_elec, nw);
    k_shell_mask<<<grid, kMaskThreads, sizeof(uint32_t) * mw, st>>>(s, mt.Qhi, mt.atom_R2f, mt.sh_R2f, R, mw, masks);
    return cudaGetLastError();
}

template <int NQ, int G>
static cudaError_t launch_c15_nq(const C15Args &a, int nwarps, cudaStream_t st)
{
    const size_t sm = sizeof(float4) * G * kC15Chunk + sizeof(double) * kC15Warps * G * 64 +
                      sizeof(uint32_t) * (G + 1) * a.mw + sizeof(int) * ((size_t)a.s.n_ao + 2);
    cudaError_t e = cudaFuncSetAttribute(k_c15_ff<NQ, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid(a.s.n_elec, (a.nw + G - 1) / G);
    k_c15_ff<NQ, G><<<grid, 32 * nwarps, sm, st>>>(a);
    return cudaGetLastError();
}

template <int G>
static cudaError_t launch_c15_g(const C15Args &a, cudaStream_t st)
{
    // the unsorted union list is staged in the AO-value buffer
    if ((size_t)a.s.n_ao > (size_t)G * kC15Chunk * 4) return cudaErrorInvalidValue;
    const int u_up = (a.s.n_up + 31) / 32, u_dn = (a.s.n_dn + 31) / 32;
    const int umax = u_up > u_dn ? u_up : u_dn;
    if (umax > 32) return cudaErrorInvalidValue;          // more than 1024 orbitals per spin
    const int nwarps = umax < kC15Warps ? (umax > 0 ? umax : 1) : kC15Warps;
    switch (umax / nwarps) {
    case 0:
    case 1: return launch_c15_nq<1, G>(a, nwarps, st);
    case 2: return launch_c15_nq<2, G>(a, nwarps, st);
    case 3: return launch_c15_nq<3, G>(a, nwarps, st);
    case 4:
        if constexpr (G <= 2) return launch_c15_nq<4, G>(a, nwarps, st);
        else return launch_c15_g<2>(a, st);           // 4 units x 4 walkers would not fit the registers
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_c15_ff(const SysDev &s, const FfBasis &fb, int nw, const double *R, const uint32_t *masks,
                          int mw, const float2 *const *A, const int *ns32, const float *const *cmax,
                          double *X, double *L5, cudaStream_t st, int walkers_per_cta)
{
    if (nw == 0) return cudaSuccess;
    C15Args a;
    a.s = s; a.fb = fb; a.nw = nw; a.mw = mw; a.R = R; a.masks = masks;
    for (int spin = 0; spin < 2; ++spin) { a.A[spin] = A[spin]; a.ns32[spin] = ns32[spin]; a.cmax[spin] = cmax[spin]; }
    a.X = X; a.L5 = L5;
    switch (walkers_per_cta) {
    case 2: return launch_c15_g<2>(a, st);
    case 4: return launch_c15_g<4>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

size_t tc_smem_bytes(const SysDev &s, int mw)
{
    return 1024 + kTcSmemFixed + sizeof(uint32_t) * TC_M * (size_t)mw + sizeof(int) * ((size_t)s.n_ao + TC_K);
}

cudaError_t launch_tc_contract(const SysDev &s, int nw, const double *R, const uint32_t *masks, int mw,
                               const TcTables &tt, float *Cg, uint32_t *wstatus, cudaStream_t st, const WaitCfg &wc)
{
    if (nw == 0) return cudaSuccess;
    TcArgs a;
    a.s = s; a.R = R; a.masks = masks; a.mw = mw; a.nw = nw;
    a.tt = tt;
    a.Cg = Cg; a.wstatus = wstatus;
    a.wait_ns = wc.limit_ns;
    const size_t sm = tc_smem_bytes(s, mw);
    if (sm > 227 * 1024) return cudaErrorInvalidConfiguration;   // system too large for one tile
    cudaError_t e = cudaFuncSetAttribute(k_tc_contract, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int nmax = s.n_up > s.n_dn ? s.n_up : s.n_dn;
    dim3 grid((nmax + TC_N - 1) / TC_N, s.n_elec, (nw + TC_M - 1) / TC_M);
    k_tc_contract<<<grid, kTcThreads, sm, st>>>(a);
    return cudaGetLastError();
}

__global__ void k_widen(const float *__restrict__ src, size_t spitch, double *__restrict__ dst, size_t dpitch,
                        size_t width)
{
    const float *srow = src + (size_t)blockIdx.y * spitch;
    double *drow = dst + (size_t)blockIdx.y * dpitch;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < width; q += (size_t)gridDim.x * blockDim.x)
        drow[q] = (double)srow[q];
}

// rows x width elements, pitches in elements
cudaError_t launch_widen(const float *src, size_t spitch, double *dst, size_t dpitch, size_t width, int rows,
                         cudaStream_t st)
{
    if (rows == 0 || width == 0) return cudaSuccess;
    dim3 grid((unsigned)((width + 255) / 256 < 1024 ? (width + 255) / 256 : 1024), rows);
    k_widen<<<grid, 256, 0, st>>>(src, spitch, dst, dpitch, width);
    return cudaGetLastError();
}

}  // namespace qmc
