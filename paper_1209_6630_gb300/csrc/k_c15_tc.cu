// Steps a2+a3 of the mixed path for C1 (the Slater matrix) and C5 (its
// Laplacian companion) on the tcgen05 tensor cores, at the accuracy the
// float-float kernel gives (~2^-40 normwise), from exact BF16 slices.
//
// Splitting (error-free, in the manner of Ozaki's scheme): with E_w the
// exponent bound of walker row w (|b| < 2^E_w over its AOs) and F_k that of MO
// column k (|A| < 2^F_k),
//   b = 2^E_w sum_i s_i,   A = 2^F_k sum_j t_j,   s_i, t_j = integer 2^(-7 (i+1))
// with |integer| <= 128 (i = 0) or about 64 (i >= 1), six slices each (42
// bits).  Every slice is exact in BF16, every product s_i t_j exact in FP32,
// and a sum over K AOs of the products with the same i + j = d is an integer
// multiple of 2^(-7 (d+2)) of at most 20865 K units (d <= 2): the FP32
// tensor-core accumulator holds it exactly for K <= 804; in the chunks of
// 1024 AOs it can pass 2^24 units only with more than ~800 terms near the
// row and column maxima of equal sign, and is then rounded by one unit.
// Four accumulators per output: d = 0, 1, 2 and d = 3..5 together (its
// rounding is 2^-45 of the result); pairs with d > 5 are dropped (< 2^-42).  The epilogue adds the
// four in FP64 and scales by 2^(E_w + F_k).
//
// k_c15_prep (one CTA per electron and tile of 128 walkers): the union AO
// list of the tile (as in k_tc_contract), a first pass in FP32 for the row
// bounds E_w of the values and of the Laplacians, then float-float AO values
// and Laplacians (as in k_c15_ff), sliced and written as 12 operand planes
// per K step of 64 AOs ([output][slice], K-major 128-byte swizzle, the
// layout the MMA reads) to a staging buffer in HBM.
//
// The producer's FP32 pass also evaluates the AO gradients and writes them as
// FP16 (or BF16) hi/lo planes scaled by exact powers of two, the operands of
// C2..C4 (three products hi.hi + hi.lo + lo.hi per output, FP32 accumulation,
// as in k_tc_contract), so the gradients are evaluated once per (electron,
// walker tile) instead of once per MO tile.
//
// k_c15_mma (one CTA per MO tile of 128, walker tile, electron and output
// class: C1, C5, or C2..C4 together):
// per stage of 32 AOs, the 6 slice planes of its output (one bulk copy) and
// the 6 slice planes of the MO coefficient rows gathered by AO index
// (MN-major, cp.async) from copy warps; a converged MMA warp issues the 21
// slice-pair MMAs of each K16 sub-step into the four TMEM accumulators and
// commits to mbarriers; waits are bounded by %globaltimer
// (QMC_STATUS_TIMEOUT on expiry).  Unions longer than 1024 AOs
// are accumulated in chunks of 1024, each added to the output in FP64.
#include "ao_ff.cuh"
#include "qmc_internal.cuh"
#include "slices.cuh"
#include "umma.cuh"

namespace qmc {

constexpr int kPrepThreads = 256;                              // two threads per walker row
constexpr int kMmaEpWarps = 8;                                 // MMA kernel: epilogue warps,
constexpr int kMmaCpWarps = 4;                                 // copy warps
constexpr int kMmaThreads = 32 * (kMmaEpWarps + kMmaCpWarps + 1);   // and an MMA warp
constexpr int kGradPlane0 = 2 * kC15Slices;                    // first C2..C4 plane of a stage
constexpr int kPlanesPerStep = 2 * kC15Slices + 6;             // [C1 slice][C5 slice][gradient l][hi, lo]
// A K step of 64 AOs is staged as two stages of 32 (the MMA kernel double-buffers
// stages): per stage and plane [128 rows][32 K] 16-bit, K-major, 64-byte swizzle.
constexpr int SK = 32;
constexpr uint32_t kSPlaneBytes = TC_M * SK * 2;               // 8 KB
constexpr uint32_t kSBPlaneBytes = SK * TC_N * 2;              // 8 KB, MN-major, 128-byte swizzle
constexpr size_t kStageBytes = (size_t)kPlanesPerStep * kSPlaneBytes;
constexpr size_t kStepBytes = 2 * kStageBytes;
constexpr int kChunkSteps = 16;                                // 1024 AOs per exact accumulation
constexpr int kAcc = 4;                                        // accumulators per output

struct C15TcArgs {
    SysDev s;
    FfBasis fb;
    const float *pgf, *pcf, *scf, *Qhi, *Qlo;
    const double *R;
    const uint32_t *masks;
    int mw, nw;
    int e0;                        // first electron of the batch
    int n_tiles;                   // walker tiles of 128
    int kmax_steps;                // staging capacity per (electron, tile), in K steps
    unsigned char *planes;         // [batch e][tile][kmax_steps][12][16 KB]
    int *ao_list;                  // [batch e][tile][kmax_steps * 64]
    int *nks;                      // [batch e][tile]
    int *rexp;                     // [batch e][tile][128][2]
    const uint16_t *slice[2];
    const int *fexp[2];
    int ns_pad[2];
    double *X, *L5;
    float *Cg;                     // C2..C4, FP32 [W][3][...]
    TcTables tt;
    uint32_t *wstatus;
    unsigned long long wait_ns;    // limit of each wait (WaitCfg)
    int expire_tile;               // test hook: walker tile whose first CTA's wait runs out (-1: none)
    int c1_only;                   // the C-free variant: C1 alone (value planes only, MMA class C1 only)
};

// Radial part and AO value / Laplacian in FP32 (for the row bounds only).
struct F32Radial {
    float dx, dy, dz, g, gd, gl;
};

__device__ __forceinline__ void f32_radial(const SysDev &s, const C15TcArgs &a, int sh, float rxh, float rxl,
                                           float ryh, float ryl, float rzh, float rzl, F32Radial &o)
{
    const int at = s.sh_atom[sh];
    o.dx = (rxh - a.Qhi[3 * at]) + (rxl - a.Qlo[3 * at]);
    o.dy = (ryh - a.Qhi[3 * at + 1]) + (ryl - a.Qlo[3 * at + 1]);
    o.dz = (rzh - a.Qhi[3 * at + 2]) + (rzl - a.Qlo[3 * at + 2]);
    const float d2 = o.dx * o.dx + o.dy * o.dy + o.dz * o.dz;
    float g = 0.f, gd = 0.f, gl = 0.f;
    const int p0 = s.sh_pstart[sh], np = s.sh_nprim[sh];
    for (int p = 0; p < np; ++p) {
        const float gam = a.pgf[p0 + p];
        const float ce = a.pcf[p0 + p] * expf(-gam * d2);
        g += ce;
        gd += gam * ce;
        gl += (4.f * gam * d2 - 6.f) * gam * ce;
    }
    o.g = g;
    o.gd = gd;
    o.gl = gl;
}

__device__ __forceinline__ void f32_angular(const SysDev &s, const C15TcArgs &a, int mu, const F32Radial &rd,
                                            float &v, float &lp, float &g1, float &g2, float &g3)
{
    const int pw = s.ao_pow[mu];
    const int nx = pw & 255, ny = (pw >> 8) & 255, nz = (pw >> 16) & 255;
    auto ip = [](float x, int n) {
        float y = 1.f;
        for (int i = 0; i < n; ++i) y *= x;
        return y;
    };
    const float px = ip(rd.dx, nx), py = ip(rd.dy, ny), pz = ip(rd.dz, nz);
    const float P = px * py * pz;
    const float dpx = nx ? nx * ip(rd.dx, nx - 1) : 0.f;
    const float dpy = ny ? ny * ip(rd.dy, ny - 1) : 0.f;
    const float dpz = nz ? nz * ip(rd.dz, nz - 1) : 0.f;
    const float ddx = nx > 1 ? nx * (nx - 1) * ip(rd.dx, nx - 2) : 0.f;
    const float ddy = ny > 1 ? ny * (ny - 1) * ip(rd.dy, ny - 2) : 0.f;
    const float ddz = nz > 1 ? nz * (nz - 1) * ip(rd.dz, nz - 2) : 0.f;
    const float c = a.scf[mu];
    const float m2gd = -2.f * rd.gd;
    v = c * P * rd.g;
    lp = c * ((ddx * py * pz + px * ddy * pz + px * py * ddz) * rd.g + P * (rd.gl - 4.f * (nx + ny + nz) * rd.gd));
    g1 = c * (dpx * py * pz * rd.g + m2gd * rd.dx * P);
    g2 = c * (px * dpy * pz * rd.g + m2gd * rd.dy * P);
    g3 = c * (px * py * dpz * rd.g + m2gd * rd.dz * P);
}

// three CTAs per SM (80 registers; a small spill costs less than the latency it hides).
// kC1Only: the C-free variant's producer: float-float values alone, six planes per stage.
template <bool kC1Only>
__global__ void __launch_bounds__(kPrepThreads, 3) k_c15_prep(C15TcArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *mask_s = reinterpret_cast<uint32_t *>(smem_raw);           // [128][mw]
    int *ao_s = reinterpret_cast<int *>(mask_s + TC_M * a.mw);           // [n_ao + 64]
    __shared__ uint32_t union_s[256];
    __shared__ int warp_s[kPrepThreads / 32];

    const SysDev &s = a.s;
    const int tile = blockIdx.x, el = blockIdx.y, e = a.e0 + el;
    const int t = threadIdx.x, row = t >> 1, half = t & 1;
    const int w = tile * TC_M + row;
    const bool wvalid = w < a.nw;
    const int mw = a.mw;
    const size_t slot = (size_t)el * a.n_tiles + tile;

    for (int q = t; q < TC_M * mw; q += kPrepThreads) {
        const int m = q / mw, j = q - m * mw;
        const int wm = tile * TC_M + m;
        mask_s[q] = (wm < a.nw) ? a.masks[((size_t)wm * s.n_elec + e) * mw + j] : 0u;
    }
    __syncthreads();
    for (int j = t; j < mw; j += kPrepThreads) {
        uint32_t u = 0;
        for (int m = 0; m < TC_M; ++m) u |= mask_s[m * mw + j];
        union_s[j] = u;
    }
    __syncthreads();
    const int K = aos_from_mask_n(s, union_s, mw, ao_s, warp_s);
    const int nks = (K + TC_K - 1) / TC_K;
    for (int q = K + t; q < nks * TC_K; q += kPrepThreads) ao_s[q] = -1;
    __syncthreads();
    int *lst = a.ao_list + slot * (size_t)a.kmax_steps * TC_K;
    for (int q = t; q < nks * TC_K; q += kPrepThreads) lst[q] = ao_s[q];
    if (t == 0) a.nks[slot] = nks;

    const double *rw = a.R + ((size_t)(wvalid ? w : 0) * s.n_elec + e) * 3;
    const float2 r2[3] = {ff::from_double(rw[0]), ff::from_double(rw[1]), ff::from_double(rw[2])};
    const uint32_t *my_mask = mask_s + row * mw;
    auto active = [&](int mu, int &sh) {
        if (mu < 0 || !wvalid) return false;
        sh = s.ao_shell[mu];
        return ((my_mask[sh >> 5] >> (sh & 31)) & 1u) != 0;
    };

    unsigned char *pl = a.planes + slot * (size_t)a.kmax_steps * kStepBytes;
    // pass 1 (FP32; radial part once per shell): bounds of |value| and
    // |Laplacian| over the row, and the gradient planes of C2..C4
    float vmax = 0.f, lmax = 0.f;
    if constexpr (kC1Only) {
        F32Radial rd;
        int last_sh = -1;
        for (int ks = 0; ks < nks; ++ks)
            for (int q = half * 32; q < half * 32 + 32; ++q) {
                const int mu = ao_s[ks * TC_K + q];
                int sh;
                if (!active(mu, sh)) continue;
                if (sh != last_sh) {
                    last_sh = sh;
                    f32_radial(s, a, sh, r2[0].x, r2[0].y, r2[1].x, r2[1].y, r2[2].x, r2[2].y, rd);
                }
                float v, lp, g1, g2, g3;
                f32_angular(s, a, mu, rd, v, lp, g1, g2, g3);
                vmax = fmaxf(vmax, fabsf(v));
            }
    } else {
        F32Radial rd;
        int last_sh = -1;
        const int f16 = a.tt.f16;
        for (int ks = 0; ks < nks; ++ks)
            for (int c8 = half * 4; c8 < half * 4 + 4; ++c8) {
                float gv[3][8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    gv[0][q] = gv[1][q] = gv[2][q] = 0.f;
                    const int mu = ao_s[ks * TC_K + c8 * 8 + q];
                    int sh;
                    if (!active(mu, sh)) continue;
                    if (sh != last_sh) {
                        last_sh = sh;
                        f32_radial(s, a, sh, r2[0].x, r2[0].y, r2[1].x, r2[1].y, r2[2].x, r2[2].y, rd);
                    }
                    float v, lp;
                    f32_angular(s, a, mu, rd, v, lp, gv[0][q], gv[1][q], gv[2][q]);
                    vmax = fmaxf(vmax, fabsf(v));
                    lmax = fmaxf(lmax, fabsf(lp));
                }
                // stage 2 ks + c8 / 4 (this thread's half), chunk c8 % 4 within it
                const uint32_t off = a_off64(row, c8 & 3);
                unsigned char *stp = pl + (size_t)(2 * ks + (c8 >> 2)) * kStageBytes +
                                     (size_t)kGradPlane0 * kSPlaneBytes;
#pragma unroll
                for (int l = 0; l < 3; ++l) {
                    uint32_t hi[4], lo[4];
                    const float isc = a.tt.in_scale[l];
#pragma unroll
                    for (int q = 0; q < 4; ++q) split2(gv[l][2 * q] * isc, gv[l][2 * q + 1] * isc, f16, hi[q], lo[q]);
                    *reinterpret_cast<uint4 *>(stp + (size_t)(2 * l) * kSPlaneBytes + off) =
                        make_uint4(hi[0], hi[1], hi[2], hi[3]);
                    *reinterpret_cast<uint4 *>(stp + (size_t)(2 * l + 1) * kSPlaneBytes + off) =
                        make_uint4(lo[0], lo[1], lo[2], lo[3]);
                }
            }
    }
    vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, 1));
    lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, 1));
    const int Ev = exp_bound(vmax), El = exp_bound(lmax);
    if (half == 0) {
        a.rexp[(slot * TC_M + row) * 2] = Ev;
        a.rexp[(slot * TC_M + row) * 2 + 1] = El;
    }

    if constexpr (kC1Only) {
        for (int ks = 0; ks < nks; ++ks)
            for (int c8 = half * 4; c8 < half * 4 + 4; ++c8) {
                uint32_t wv[kC15Slices][4];
#pragma unroll
                for (int q2 = 0; q2 < 4; ++q2) {
                    float sv[2][kC15Slices];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int mu = ao_s[ks * TC_K + c8 * 8 + 2 * q2 + h];
                        int sh;
                        const float2 v = active(mu, sh) ? ao_val_ff(s, a.fb, mu, r2) : make_float2(0.f, 0.f);
                        slice6(v, Ev, sv[h]);
                    }
#pragma unroll
                    for (int j = 0; j < kC15Slices; ++j) wv[j][q2] = bf16_pair(sv[0][j], sv[1][j]);
                }
                const uint32_t off = a_off64(row, c8 & 3);
                unsigned char *stp = pl + (size_t)(2 * ks + (c8 >> 2)) * kStageBytes;
#pragma unroll
                for (int j = 0; j < kC15Slices; ++j)
                    *reinterpret_cast<uint4 *>(stp + (size_t)j * kSPlaneBytes + off) =
                        make_uint4(wv[j][0], wv[j][1], wv[j][2], wv[j][3]);
            }
        return;
    }
    // pass 2: float-float values and Laplacians, sliced into the operand planes
    // (the float-float radial part is recomputed per AO here: caching it per shell,
    // as in pass 1, keeps 12 more registers live across the slicing and measured slower)
    for (int ks = 0; ks < nks; ++ks)
        for (int c8 = half * 4; c8 < half * 4 + 4; ++c8) {
            uint32_t wv[kC15Slices][4], wl[kC15Slices][4];
#pragma unroll
            for (int q2 = 0; q2 < 4; ++q2) {
                float sv[2][kC15Slices], sl[2][kC15Slices];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int mu = ao_s[ks * TC_K + c8 * 8 + 2 * q2 + h];
                    int sh;
                    float2 v = make_float2(0.f, 0.f), lp = make_float2(0.f, 0.f);
                    if (active(mu, sh)) ao_val_lap_ff(s, a.fb, mu, r2, v, lp);
                    slice6(v, Ev, sv[h]);
                    slice6(lp, El, sl[h]);
                }
#pragma unroll
                for (int j = 0; j < kC15Slices; ++j) {
                    wv[j][q2] = bf16_pair(sv[0][j], sv[1][j]);
                    wl[j][q2] = bf16_pair(sl[0][j], sl[1][j]);
                }
            }
            const uint32_t off = a_off64(row, c8 & 3);
            unsigned char *stp = pl + (size_t)(2 * ks + (c8 >> 2)) * kStageBytes;
#pragma unroll
            for (int j = 0; j < kC15Slices; ++j) {
                *reinterpret_cast<uint4 *>(stp + (size_t)j * kSPlaneBytes + off) =
                    make_uint4(wv[j][0], wv[j][1], wv[j][2], wv[j][3]);
                *reinterpret_cast<uint4 *>(stp + (size_t)(kC15Slices + j) * kSPlaneBytes + off) =
                    make_uint4(wl[j][0], wl[j][1], wl[j][2], wl[j][3]);
            }
        }
}

// Bounded wait of a whole warp, which stays converged (every lane polls; the phase, once
// complete, stays complete until this warp has moved on), with the CTA's abort flag.
__device__ __forceinline__ bool c15_wait_warp(uint32_t mbar, uint32_t parity, uint64_t limit_ns,
                                              volatile int *abort, int lane)
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

// Warp-specialised: 8 epilogue warps (TMEM lane quadrant x two groups of 64 columns), 4
// copy warps and an MMA warp.  Per stage of 32 AOs the copy warps move the 6 staged operand
// planes with one bulk copy (TMA) and gather the MO-coefficient slice rows of the stage's
// AOs with 16-byte cp.async into the MN-major, 128-byte-swizzled layout the MMA reads (AO
// padding rows and columns past the padded MO count as zeros), into one of two stage
// buffers; the MMA warp issues the stage's slice-pair MMAs (each through elect.sync) and
// releases the buffer with a commit; at the end of each chunk of 1024 AOs the epilogue adds
// the accumulators to the output.  (Gathering the rows with tensor TMA instead --
// tile::gather4, 96 copies of 4 rows x 128 bytes per stage -- was slower: the TMA unit's
// cost per copy, not the bytes, set the pace.)
__global__ void __launch_bounds__(kMmaThreads, 1) k_c15_mma(C15TcArgs a)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    unsigned char *base = tc_smem + ((1024 - (smem_u32(tc_smem) & 1023)) & 1023);
    // two stage buffers, each [A: 6 planes x 8 KB][B: 6 planes x 8 KB]
    constexpr uint32_t kBufBytes = kC15Slices * (kSPlaneBytes + kSBPlaneBytes);
    int *ao_s = reinterpret_cast<int *>(base + 2 * kBufBytes);     // [kmax_steps * 64]
    __shared__ __align__(8) uint64_t bar[6];
    __shared__ uint32_t tmem_slot;
    __shared__ int s_abort, s_never;

    const SysDev &s = a.s;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    // o: C1, C5, C2..C4 (the C-free variant: C1 alone)
    const int mt = blockIdx.x, tile = blockIdx.y;
    const int el = a.c1_only ? (int)blockIdx.z : (int)blockIdx.z / 3, o = a.c1_only ? 0 : (int)blockIdx.z % 3;
    const int e = a.e0 + el;
    const int spin = e >= s.n_up;
    const int ei = spin ? e - s.n_up : e;
    const int ns = spin ? s.n_dn : s.n_up;
    const int k0 = mt * TC_N;
    if (k0 >= ns) return;
    const int nspad = a.ns_pad[spin];
    const int ncols = min(TC_N, nspad - k0);
    const size_t slot = (size_t)el * a.n_tiles + tile;
    const int nks = a.nks[slot];
    const int *lst = a.ao_list + slot * (size_t)a.kmax_steps * TC_K;
    for (int q = t; q < nks * TC_K; q += kMmaThreads) ao_s[q] = lst[q];
    const uint32_t b0 = smem_u32(&bar[0]);
    auto FULL = [&](int buf) { return b0 + 8u * (uint32_t)buf; };            // stage copied
    auto EMPTY = [&](int buf) { return b0 + 8u * (uint32_t)(2 + buf); };     // stage's MMAs complete
    const uint32_t bCD = b0 + 32u;                                            // chunk accumulated
    const uint32_t bED = b0 + 40u;                                            // accumulators read
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;"
                     :: "r"(smem_u32(&tmem_slot)) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 32) {
        for (int b = 0; b < 2; ++b) { mbar_init(FULL(b), 1 + 32 * kMmaCpWarps); mbar_init(EMPTY(b), 1); }
        mbar_init(bCD, 1);
        mbar_init(bED, kMmaEpWarps);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
        s_never = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const bool grad = o == 2;
    const uint64_t kWait = a.wait_ns;
    const int nst = 2 * nks;                             // stages of 32 AOs
    const int nchunk = max(1, (nst + 2 * kChunkSteps - 1) / (2 * kChunkSteps));
    int nissued = 0, nmma = 0;                           // stages copied / multiplied (drain)

    if (warp >= kMmaEpWarps && warp < kMmaEpWarps + kMmaCpWarps) {
        // ---- copy warps: the stage's 6 operand planes by one bulk copy (TMA), the gathered
        // MO-coefficient rows by 16-byte cp.async; each lane waits for its own copies, makes
        // them visible to the tensor cores' proxy and arrives
        const int cl = t - 32 * kMmaEpWarps;                 // 0 .. 32 * kMmaCpWarps - 1
        const unsigned char *Ag = a.planes + slot * (size_t)a.kmax_steps * kStepBytes +
                                  (size_t)o * kC15Slices * kSPlaneBytes;     // o = 2: the gradient planes
        const int nbplanes = grad ? 2 : kC15Slices;
        const uint16_t *__restrict__ Bsl = a.slice[spin];
        const size_t slice_stride = (size_t)s.n_ao * nspad;
        for (int sg = 0; sg < nst; ++sg) {
            const int buf = sg & 1;
            if (sg >= 2 && !c15_wait_warp(EMPTY(buf), ((sg >> 1) - 1) & 1, kWait, &s_abort, lane)) break;
            unsigned char *Ab = base + buf * kBufBytes, *Bb = Ab + kC15Slices * kSPlaneBytes;
            if (cl == 0) {
                mbar_expect_tx(FULL(buf), kC15Slices * kSPlaneBytes);
                bulk_g2s(smem_u32(Ab), Ag + (size_t)sg * kStageBytes, kC15Slices * kSPlaneBytes, FULL(buf));
            }
            for (int q = cl; q < nbplanes * SK * (TC_N / 8); q += 32 * kMmaCpWarps) {
                const int j = q / (SK * (TC_N / 8));
                const int rem = q - j * (SK * (TC_N / 8));
                const int r = rem / (TC_N / 8), c = rem - r * (TC_N / 8);
                const int mu = ao_s[sg * SK + r];
                const bool v = mu >= 0 && 8 * c < ncols;
                const uint16_t *bsrc = grad ? (j ? a.tt.lo[spin] : a.tt.hi[spin]) : Bsl + j * slice_stride;
                const uint16_t *src = bsrc + (size_t)(v ? mu : 0) * nspad + k0 + (v ? 8 * c : 0);
                cp_async16(smem_u32(Bb + j * kSBPlaneBytes + b_off(r, 8 * c)), src, v);
            }
            asm volatile("cp.async.wait_all;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(FULL(buf));
            nissued = sg + 1;
        }
    } else if (warp == kMmaEpWarps + kMmaCpWarps) {
        // ---- MMA warp: converged, one elected lane issues each MMA and commit
        const uint32_t idesc = umma_idesc_f16(TC_M, ncols, grad ? (a.tt.f16 ? 0 : 1) : 1);
        for (int c = 0; c < nchunk; ++c) {
            const int s0 = c * 2 * kChunkSteps, s1 = min(nst, s0 + 2 * kChunkSteps);
            if (c > 0 && !c15_wait_warp(bED, (c - 1) & 1, kWait, &s_abort, lane)) break;
            bool ok = true;
            for (int sg = s0; sg < s1; ++sg) {
                const int buf = sg & 1;
                if (!c15_wait_warp(FULL(buf), (sg >> 1) & 1, kWait, &s_abort, lane)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                // descriptors of the buffer's first A and B planes; the others differ only in
                // the start-address field (address / 16 in the low bits), by constants
                const uint32_t a0 = smem_u32(base + buf * kBufBytes);
                const uint64_t dA = umma_desc_sw64(a0, 512);
                const uint64_t dB = umma_desc(a0 + kC15Slices * kSPlaneBytes, kBLbo, kBSbo);
                const uint32_t fresh = sg == s0 ? 1u : 0u;     // first stage of a chunk
                if (grad) {
#pragma unroll
                    for (int kk = 0; kk < SK / 16; ++kk) {
                        const uint64_t bh = dB + ((2 * kk * kBSbo) >> 4);
                        const uint64_t bl = dB + ((kSBPlaneBytes + 2 * kk * kBSbo) >> 4);
#pragma unroll
                        for (int l = 0; l < 3; ++l) {
                            const uint64_t ah = dA + (((2 * l) * kSPlaneBytes + 32 * kk) >> 4);
                            const uint64_t al = dA + (((2 * l + 1) * kSPlaneBytes + 32 * kk) >> 4);
                            const uint32_t dd = tmem + l * TC_N;
                            umma_bf16_warp(dd, ah, bh, idesc, (fresh && kk == 0) ? 0u : 1u);
                            umma_bf16_warp(dd, ah, bl, idesc, 1u);
                            umma_bf16_warp(dd, al, bh, idesc, 1u);
                        }
                    }
                } else {
#pragma unroll
                    for (int kk = 0; kk < SK / 16; ++kk) {
#pragma unroll
                        for (int d = 0; d < kC15Slices; ++d) {
                            const int acc = d < kAcc - 1 ? d : kAcc - 1;
#pragma unroll
                            for (int i = 0; i <= d; ++i) {
                                const int j = d - i;
                                const uint64_t ad = dA + ((i * kSPlaneBytes + 32 * kk) >> 4);
                                const uint64_t bd = dB + ((j * kSBPlaneBytes + 2 * kk * kBSbo) >> 4);
                                const bool first = kk == 0 && i == 0 && d <= kAcc - 1;
                                umma_bf16_warp(tmem + acc * TC_N, ad, bd, idesc, (fresh && first) ? 0u : 1u);
                            }
                        }
                    }
                }
                umma_commit_warp(EMPTY(buf));                 // the stage buffer may be refilled
                nmma = sg + 1;
            }
            if (!ok) break;
            umma_commit_warp(bCD);                            // the chunk's sums are complete
        }
    } else {
        // ---- epilogue warps: row = TMEM lane, columns cgrp * 32 + 64 m
        const size_t msz = (size_t)s.n_up * s.n_up + (size_t)s.n_dn * s.n_dn;
        double *outp = o ? a.L5 : a.X;
        const int row = (warp & 3) * 32 + lane;        // TMEM lane = walker row of this thread
        const int w = tile * TC_M + row;
        const int cgrp = warp >> 2;
        // test hook: the C1 CTA of electron 0, MO tile 0 of the chosen walker tile
        const bool expire = tile == a.expire_tile && e == 0 && mt == 0 && o == 0;
        for (int c = 0; c < nchunk; ++c) {
            bool ok;
            if (expire && c == 0) {
                int f = 0;
                if (lane == 0) {
                    f = flag_wait(&s_never, kWait);
                    if (!f) s_abort = 1;
                }
                ok = __shfl_sync(0xffffffffu, f, 0) != 0;
            } else {
                ok = c15_wait_warp(bCD, c & 1, kWait, &s_abort, lane);
            }
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int c0 = c * 2 * kChunkSteps;          // 0 for the first chunk
            if (grad) {
                // epilogue C2..C4: FP32 accumulators times the power-of-two output scale
                const size_t nss = (size_t)ns * ns;
                float *crow = a.Cg + (size_t)(w < a.nw ? w : 0) * 3 * msz +
                              (spin ? 3 * (size_t)s.n_up * s.n_up : 0) + (size_t)ei * ns;
                for (int l = 0; l < 3; ++l) {
                    const float osc = a.tt.out_scale[spin][l];
                    for (int cb = cgrp * 32; cb < ncols; cb += 32 * (kMmaEpWarps / 4)) {
                        uint32_t v[32];
                        tmem_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(l * TC_N + cb), v);
                        if (w < a.nw) {
                            float *dst = crow + (size_t)l * nss;
#pragma unroll
                            for (int q = 0; q < 32; ++q) {
                                const int k = k0 + cb + q;
                                if (k >= ns) break;
                                const float val = nks > 0 ? __uint_as_float(v[q]) * osc : 0.f;
                                if (c0 == 0) dst[k] = val;
                                else dst[k] += val;
                            }
                        }
                    }
                }
            } else {
                // epilogue C1 / C5: the four accumulators (orders 0, 1, 2 exact; 3..5 rounded at
                // 2^-45) summed as float pairs on the FP32 pipes (each addition exact but the last
                // two lo additions, 2^-47 of the sum), scaled by 2^(E_w + F_k) and converted once:
                // two conversions and one FP64 addition per element instead of nine FP64 operations
                const int E = (w < a.nw) ? a.rexp[(slot * TC_M + row) * 2 + o] : 0;
                double *dst = outp + (size_t)(w < a.nw ? w : 0) * msz + (spin ? (size_t)s.n_up * s.n_up : 0) +
                              (size_t)ei * ns;
                for (int cb = cgrp * 32; cb < ncols; cb += 32 * (kMmaEpWarps / 4)) {
                    float hs[32], ls[32];
                    {
                        uint32_t v[32];
                        tmem_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)cb, v);
#pragma unroll
                        for (int q = 0; q < 32; ++q) {
                            hs[q] = __uint_as_float(v[q]);
                            ls[q] = 0.f;
                        }
                    }
#pragma unroll
                    for (int acc = 1; acc < kAcc; ++acc) {
                        uint32_t v[32];
                        tmem_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(acc * TC_N + cb), v);
#pragma unroll
                        for (int q = 0; q < 32; ++q) {
                            float sh, se;
                            ff::two_sum(hs[q], __uint_as_float(v[q]), sh, se);
                            hs[q] = sh;
                            ls[q] = __fadd_rn(ls[q], se);
                        }
                    }
                    if (w < a.nw && nks > 0) {
#pragma unroll
                        for (int q = 0; q < 32; ++q) {
                            const int k = k0 + cb + q;
                            if (k >= ns) break;
                            float h2, l2;
                            ff::fast_two_sum(hs[q], ls[q], h2, l2);
                            const int ex = E + a.fexp[spin][k];   // exact power-of-two scaling in FP32
                            const double val = (double)scale_pow2(h2, ex) + (double)scale_pow2(l2, ex);
                            if (c0 == 0) dst[k] = val;
                            else dst[k] += val;
                        }
                    } else if (w < a.nw) {
                        for (int q = 0; q < 32 && k0 + cb + q < ns; ++q) dst[k0 + cb + q] = 0.0;
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(bED);
        }
    }
    __syncthreads();
    if (s_abort) {
        if (warp < kMmaEpWarps && (warp >> 2) == 0) {
            const int w = tile * TC_M + (warp & 3) * 32 + lane;
            if (w < a.nw) atomicOr(a.wstatus + w, (uint32_t)QMC_STATUS_TIMEOUT);
        }
        // nothing may land in shared memory or TMEM after the CTA exits
        if (warp == kMmaEpWarps && lane == 0)              // the bulk copies (cp.async: waited above)
            for (int sg = max(0, nissued - 2); sg < nissued; ++sg) mbar_wait(FULL(sg & 1), (sg >> 1) & 1, kDrainNs);
    }
    if (warp == kMmaEpWarps + kMmaCpWarps && lane == 0)
        for (int sg = max(0, nmma - 2); sg < nmma; ++sg) mbar_wait(EMPTY(sg & 1), (sg >> 1) & 1, kDrainNs);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" :: "r"(tmem) : "memory");
}

bool c15tc_fits(const SysDev &s, int mw)
{
    const int nmax = s.n_up > s.n_dn ? s.n_up : s.n_dn;
    const size_t kmax = (size_t)(s.n_ao + TC_K - 1) / TC_K;
    const size_t sm_mma = 1024 + 2 * (size_t)kC15Slices * (kSPlaneBytes + kSBPlaneBytes) + sizeof(int) * kmax * TC_K;
    const size_t sm_prep = sizeof(uint32_t) * TC_M * (size_t)mw + sizeof(int) * ((size_t)s.n_ao + TC_K);
    return nmax <= 1024 && mw <= 256 && sm_mma <= 227 * 1024 && sm_prep <= 227 * 1024;
}

// Electrons per producer / MMA launch pair: enough CTAs per launch for large
// batches of walkers (fewer launches, so fewer partly filled last waves), a
// small staging buffer for small ones; spread evenly over the launches.
size_t c15tc_batch(int n_elec, int n_tiles)
{
    const int b = n_tiles >= 8 ? 128 : (n_tiles >= 2 ? 32 : 16);
    if (n_elec <= b) return (size_t)(n_elec > 0 ? n_elec : 1);
    const int nl = (n_elec + b - 1) / b;                   // launches, then the electrons spread evenly
    return (size_t)((n_elec + nl - 1) / nl);
}

size_t c15tc_bytes(const SysDev &s, int nw)
{
    const size_t tiles = (size_t)(nw + TC_M - 1) / TC_M;
    const size_t kmax = (size_t)(s.n_ao + TC_K - 1) / TC_K;
    const size_t per = kmax * kStepBytes + kmax * TC_K * 4 + 4 + TC_M * 2 * 4;
    return c15tc_batch(s.n_elec, (int)tiles) * tiles * per + 4096;
}

cudaError_t launch_c15_tc(const SysDev &s, const FfBasis &fb, const MixedTables &mt, const TcTables &tt, int nw,
                          const double *R, const uint32_t *masks, int mw, double *X, double *L5, float *Cg,
                          uint32_t *wstatus, void *scratch, cudaStream_t st, const WaitCfg &wc, bool c1_only)
{
    if (nw == 0) return cudaSuccess;
    const int nmax = s.n_up > s.n_dn ? s.n_up : s.n_dn;
    if (nmax > 1024 || mw > 256) return cudaErrorInvalidValue;
    C15TcArgs a;
    a.s = s; a.fb = fb;
    a.pgf = mt.pgf; a.pcf = mt.pcf; a.scf = mt.scf; a.Qhi = mt.Qhi; a.Qlo = mt.Qlo;
    a.R = R; a.masks = masks; a.mw = mw; a.nw = nw;
    a.n_tiles = (nw + TC_M - 1) / TC_M;
    a.kmax_steps = (s.n_ao + TC_K - 1) / TC_K;
    const size_t nb = c15tc_batch(s.n_elec, a.n_tiles);
    char *p = static_cast<char *>(scratch);
    const size_t ntl = nb * a.n_tiles;
    a.planes = reinterpret_cast<unsigned char *>(p);
    p += ntl * a.kmax_steps * kStepBytes;
    a.ao_list = reinterpret_cast<int *>(p);
    p += ntl * a.kmax_steps * TC_K * 4;
    a.nks = reinterpret_cast<int *>(p);
    p += ((ntl * 4 + 255) / 256) * 256;
    a.rexp = reinterpret_cast<int *>(p);
    for (int spin = 0; spin < 2; ++spin) {
        a.slice[spin] = mt.slice[spin];
        a.fexp[spin] = mt.fexp[spin];
        a.ns_pad[spin] = mt.ns_pad[spin];
    }
    a.X = X; a.L5 = L5; a.Cg = Cg; a.tt = tt; a.wstatus = wstatus;
    a.wait_ns = wc.limit_ns;
    a.c1_only = c1_only ? 1 : 0;
    a.expire_tile = (wc.expire_kernels & QMC_EXPIRE_C15) && wc.expire_w >= 0 && wc.expire_w < nw ? wc.expire_w / TC_M : -1;
    const size_t sm_prep = sizeof(uint32_t) * TC_M * (size_t)mw + sizeof(int) * ((size_t)s.n_ao + TC_K);
    const size_t sm_mma = 1024 + 2 * (size_t)kC15Slices * (kSPlaneBytes + kSBPlaneBytes) +
                          sizeof(int) * (size_t)a.kmax_steps * TC_K;
    if (sm_mma > 227 * 1024 || sm_prep > 227 * 1024) return cudaErrorInvalidConfiguration;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(c1_only ? k_c15_prep<true> : k_c15_prep<false>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_prep)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_c15_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_mma)) !=
        cudaSuccess)
        return e;
    const int mtiles = (nmax + TC_N - 1) / TC_N;
    for (int e0 = 0; e0 < s.n_elec; e0 += (int)nb) {
        const int ne = s.n_elec - e0 < (int)nb ? s.n_elec - e0 : (int)nb;
        a.e0 = e0;
        if (c1_only) k_c15_prep<true><<<dim3(a.n_tiles, ne), kPrepThreads, sm_prep, st>>>(a);
        else k_c15_prep<false><<<dim3(a.n_tiles, ne), kPrepThreads, sm_prep, st>>>(a);
        k_c15_mma<<<dim3(mtiles, a.n_tiles, (c1_only ? 1 : 3) * ne), kMmaThreads, sm_mma, st>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace qmc
