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
// per K step, the 6 slice planes of its output (copied with cp.async) and the
// 6 slice planes of the MO coefficient rows gathered by AO index (MN-major);
// one thread issues the 21 slice-pair MMAs of each K16 sub-step into the four
// TMEM accumulators and commits to an mbarrier; waits are bounded by
// %globaltimer (QMC_STATUS_TIMEOUT on expiry).  Unions longer than 1024 AOs
// are accumulated in chunks of 1024, each added to the output in FP64.
#include "ao_ff.cuh"
#include "qmc_internal.cuh"
#include "slices.cuh"
#include "umma.cuh"

namespace qmc {

constexpr int kPrepThreads = 256;                              // two threads per walker row
constexpr int kMmaThreads = 512;
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

__global__ void __launch_bounds__(kMmaThreads, 1) k_c15_mma(C15TcArgs a)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    unsigned char *base = tc_smem + ((1024 - (smem_u32(tc_smem) & 1023)) & 1023);
    // two stage buffers, each [A: 6 planes x 8 KB][B: 6 planes x 8 KB]
    constexpr uint32_t kBufBytes = kC15Slices * (kSPlaneBytes + kSBPlaneBytes);
    int *ao_s = reinterpret_cast<int *>(base + 2 * kBufBytes);     // [kmax_steps * 64]
    __shared__ __align__(8) uint64_t mbar[2];
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
    if (t == 0) { s_abort = 0; s_never = 0; }

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;"
                     :: "r"(smem_u32(&tmem_slot)) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t mbs[2] = {smem_u32(&mbar[0]), smem_u32(&mbar[1])};
    const bool grad = o == 2;
    const uint32_t idesc = umma_idesc_f16(TC_M, ncols, grad ? (a.tt.f16 ? 0 : 1) : 1);
    const uint64_t kWait = a.wait_ns;
    // test hook: the C1 CTA of electron 0, MO tile 0 of the chosen walker tile
    const bool expire = tile == a.expire_tile && e == 0 && mt == 0 && o == 0;
    const uint16_t *__restrict__ Bsl = a.slice[spin];
    const unsigned char *Ag = a.planes + slot * (size_t)a.kmax_steps * kStepBytes +
                              (size_t)o * kC15Slices * kSPlaneBytes;     // o = 2: the gradient planes
    const size_t slice_stride = (size_t)s.n_ao * nspad;
    const int nbplanes = grad ? 2 : kC15Slices;
    int ncb[2] = {0, 0};                                 // commits per stage buffer
    bool ok = true;

    const size_t msz = (size_t)s.n_up * s.n_up + (size_t)s.n_dn * s.n_dn;
    double *outp = o ? a.L5 : a.X;
    const int row = (warp & 3) * 32 + lane;            // TMEM lane = walker row of this thread
    const int w = tile * TC_M + row;

    // copies of stage sg (AO positions 32 sg .. 32 sg + 31) into stage buffer buf
    auto issue_loads = [&](int sg, int buf) {
        unsigned char *Ab = base + buf * kBufBytes, *Bb = Ab + kC15Slices * kSPlaneBytes;
        const unsigned char *ag = Ag + (size_t)sg * kStageBytes;
        for (int q = t; q < kC15Slices * (int)kSPlaneBytes / 16; q += kMmaThreads)
            cp_async16(smem_u32(Ab + 16 * q), ag + 16 * (size_t)q, true);
        for (int q = t; q < nbplanes * SK * (TC_N / 8); q += kMmaThreads) {
            const int j = q / (SK * (TC_N / 8));
            const int rem = q - j * (SK * (TC_N / 8));
            const int r = rem / (TC_N / 8), c = rem - r * (TC_N / 8);
            const int mu = ao_s[sg * SK + r];
            const bool v = mu >= 0 && 8 * c < ncols;
            const uint16_t *bsrc = grad ? (j ? a.tt.lo[spin] : a.tt.hi[spin]) : Bsl + j * slice_stride;
            const uint16_t *src = bsrc + (size_t)(v ? mu : 0) * nspad + k0 + (v ? 8 * c : 0);
            cp_async16(smem_u32(Bb + j * kSBPlaneBytes + b_off(r, 8 * c)), src, v);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };

    const int nst = 2 * nks;                             // stages of 32 AOs
    for (int s0 = 0; s0 < max(nst, 1); s0 += 2 * kChunkSteps) {
        const int s1 = min(nst, s0 + 2 * kChunkSteps);
        const int c0 = s0;                               // 0 for the first chunk
        if (s0 < s1) issue_loads(s0, s0 & 1);
        for (int sg = s0; sg < s1; ++sg) {
            const int buf = sg & 1;
            if (sg + 1 < s1) {
                const int nb = buf ^ 1;
                // the MMAs of stage sg - 1 read buffer nb: wait before overwriting it
                if (ncb[nb] > 0 && !mbar_wait(mbs[nb], (ncb[nb] - 1) & 1, kWait)) s_abort = 1;
                issue_loads(sg + 1, nb);
                asm volatile("cp.async.wait_group 1;" ::: "memory");
            } else {
                asm volatile("cp.async.wait_group 0;" ::: "memory");
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (s_abort) break;
            if (t == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                // descriptors of the buffer's first A and B planes; the others differ only in
                // the start-address field (address / 16 in the low bits), by constants
                const uint32_t a0 = smem_u32(base + buf * kBufBytes);
                const uint64_t dA = umma_desc_sw64(a0, 512);
                const uint64_t dB = umma_desc(a0 + kC15Slices * kSPlaneBytes, kBLbo, kBSbo);
                const bool fresh = sg == s0;                  // first stage of a chunk
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
                            umma_bf16(dd, ah, bh, idesc, (!fresh || kk > 0) ? 1u : 0u);
                            umma_bf16(dd, ah, bl, idesc, 1u);
                            umma_bf16(dd, al, bh, idesc, 1u);
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
                                const bool first = fresh && kk == 0 && i == 0 && d <= kAcc - 1;
                                umma_bf16(tmem + acc * TC_N, ad, bd, idesc, first ? 0u : 1u);
                            }
                        }
                    }
                }
                umma_commit(mbs[buf]);
            }
            ++ncb[buf];
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        if (expire && !flag_wait(&s_never, kWait)) s_abort = 1;
        for (int bq = 0; bq < 2; ++bq)
            if (!s_abort && ncb[bq] > 0 && !mbar_wait(mbs[bq], (ncb[bq] - 1) & 1, kWait)) s_abort = 1;
        __syncthreads();
        ok = !s_abort;
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (grad) {
            // epilogue C2..C4: FP32 accumulators times the power-of-two output scale
            const size_t nss = (size_t)ns * ns;
            float *crow = a.Cg + (size_t)(w < a.nw ? w : 0) * 3 * msz +
                          (spin ? 3 * (size_t)s.n_up * s.n_up : 0) + (size_t)ei * ns;
            for (int l = 0; l < 3; ++l) {
                const float osc = a.tt.out_scale[spin][l];
                for (int cb = (warp >> 2) * 32; cb < ncols; cb += 32 * (kMmaThreads / 128)) {
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
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            continue;
        }
        // epilogue C1 / C5: the four accumulators (orders 0, 1, 2 exact; 3..5 rounded at
        // 2^-45) summed as float pairs on the FP32 pipes (each addition exact but the last
        // two lo additions, 2^-47 of the sum), scaled by 2^(E_w + F_k) and converted once:
        // two conversions and one FP64 addition per element instead of nine FP64 operations
        const int E = (w < a.nw) ? a.rexp[(slot * TC_M + row) * 2 + o] : 0;
        double *dst = outp + (size_t)(w < a.nw ? w : 0) * msz + (spin ? (size_t)s.n_up * s.n_up : 0) +
                      (size_t)ei * ns;
        for (int cb = (warp >> 2) * 32; cb < ncols; cb += 32 * (kMmaThreads / 128)) {
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
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (!ok) {
        if (w < a.nw && (warp >> 2) == 0) atomicOr(a.wstatus + w, (uint32_t)QMC_STATUS_TIMEOUT);
        asm volatile("cp.async.wait_all;" ::: "memory");
        for (int bq = 0; bq < 2; ++bq)                  // let MMAs in flight drain
            if (ncb[bq] > 0) mbar_wait(mbs[bq], (ncb[bq] - 1) & 1, kDrainNs);
    }
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
// batches of walkers, a small staging buffer for small ones.
size_t c15tc_batch(int n_elec, int n_tiles)
{
    const int b = n_tiles >= 8 ? 64 : (n_tiles >= 2 ? 32 : 16);
    return (size_t)(n_elec < b ? (n_elec > 0 ? n_elec : 1) : b);
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
