// The C-free variant of steps a3 + a5 (drift and Laplacian without the
// gradient and Laplacian matrices C2..C5).  From the cofactor identities of
// Sec. II.C (the two vector products) and the MO expansion Eq. (mo):
//   drift_{e,l} = sum_k (D^-1)_{ek} d_l phi_k(r_e) = sum_mu v_{e mu} d_l chi_mu(r_e)
//   lap_e       = sum_k (D^-1)_{ek} lap phi_k(r_e) = sum_mu v_{e mu} lap chi_mu(r_e)
//   v_{e mu}    = sum_k (D^-1)_{ek} a_{k mu}              (v_e = D^-1[e,:] A^T)
// with mu over the AOs that are not screened out for r_e.  Only C1 is formed
// (for the determinant and D^-1); the product v costs sum_s N_s^2 Kbar
// multiply-adds, against 4 sum_s N_s^2 Kbar for C2..C5.
//
// k_vd_rowexp: the exponent bound E of every D^-1 row (|D^-1[e,k]| < 2^E).
// k_vd_mma (one CTA per walker tile of 128 and electron e): the union of the
// tile's active AOs for e (from the shell masks), then per AO tile of 64: v
// on the tcgen05 tensor cores as M = 128 walkers x N = 64 AOs x K = N_s MOs
// from exact BF16 slices, the split of the C1 products (k_c15_tc.cu) with
// the roles of the indices exchanged: D^-1 rows scaled by 2^-E_{w,e} (sliced
// from the FP64 inverse once per CTA into a staging image in global memory
// that every AO tile copies), A rows scaled by 2^-G_mu (sliced at load), six
// slices each, the 21 slice pairs of order <= 5 into four FP32
// accumulators (orders 0, 1, 2 exact; 3..5 together); K stages of 32 MOs
// through one stage buffer per CTA, two CTAs per SM (the staged D^-1 slices
// by one bulk copy, the B rows by cp.async), a converged warp issuing the MMAs
// through elect.sync, mbarrier commits, bounded waits.  Epilogue:
// v = 2^(E + G_mu) (acc0 + acc1 + acc2 + acc3) as a float pair (the order sums
// are exact integers in their units; the power of two is applied exactly),
// and for every active AO of the walker the gradient (FP32) and Laplacian
// (float-float, radial part once per shell) of the AO at r_e, multiplied by v
// and accumulated as float pairs on the FP32 pipes.
// Output vd[w][e] = (drift_x, drift_y, drift_z, lap_e).
#include "ao_ff.cuh"
#include "qmc_internal.cuh"
#include "slices.cuh"
#include "umma.cuh"

namespace qmc {

namespace {

constexpr int kVdThreads = 256;
constexpr int kVdK = 32;                                      // MOs per stage
constexpr int kVdN = 64;                                      // AOs per tile (TMEM columns per accumulator)
constexpr uint32_t kVdPlane = TC_M * kVdK * 2;                // A: [128 rows][32 K] 16-bit, 64-byte swizzle: 8 KB
constexpr uint32_t kVdBPlane = kVdN * kVdK * 2;               // B: [64 rows][32 K]: 4 KB
constexpr uint32_t kVdBuf = kC15Slices * (kVdPlane + kVdBPlane);   // 6 A planes + 6 B planes: 72 KB
constexpr int kVdAcc = 4;

struct VdArgs {
    SysDev s;
    FfBasis fb;
    const double *R;
    const uint32_t *masks;
    int mw, nw;
    const double *Dinv;            // [nw][msz] rows = electrons
    size_t msz;
    const int *rexp;               // [nw][N] row exponents of D^-1
    const uint16_t *rslice[2];     // [6][n_ao][ns_pad]
    const int *gexp[2];            // [n_ao]
    int ns_pad[2];
    double *vd;                    // [nw][N][4]
    uint32_t *wstatus;
    unsigned long long wait_ns;
    const float *pgf, *pcf, *scf;  // FP32 exponents, coefficients [n_prim], AO scales [n_ao]
    const float *Qhi, *Qlo;        // nuclear positions as float pairs [n_atom][3]
    int e0;                        // first electron of this launch's batch
    unsigned char *astage;         // per CTA of the batch: the sliced D^-1 rows, one A image per K stage
    size_t astage_per;             // bytes per CTA
};

__global__ void k_vd_rowexp(int nw, int n_up, int n_dn, size_t msz, const double *__restrict__ Dinv,
                            int *__restrict__ rexp)
{
    const int N = n_up + n_dn;
    const size_t row = blockIdx.x * (size_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= (size_t)nw * N) return;
    const int w = (int)(row / N), e = (int)(row - (size_t)w * N);
    const int spin = e >= n_up, ns = spin ? n_dn : n_up, ei = spin ? e - n_up : e;
    const double *d = Dinv + (size_t)w * msz + (spin ? (size_t)n_up * n_up : 0) + (size_t)ei * ns;
    float m = 0.f;
    for (int k = lane; k < ns; k += 32) m = fmaxf(m, fabsf((float)d[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) rexp[row] = exp_bound(m);
}

// Two CTAs per SM (256 threads, N = 64 AOs per tile, one operand stage of
// 72 KB, 256 TMEM columns each): one CTA's epilogue (the AO derivatives, the
// larger part of the work) runs while the other's copies and MMAs proceed.
__global__ void __launch_bounds__(kVdThreads, 2) k_vd_mma(VdArgs a)
{
    extern __shared__ __align__(1024) unsigned char vd_smem[];
    unsigned char *base = vd_smem + ((1024 - (smem_u32(vd_smem) & 1023)) & 1023);
    int *ao_s = reinterpret_cast<int *>(base + kVdBuf);       // [n_ao + kVdN]
    __shared__ uint32_t un_s[256];
    __shared__ int warp_s[kVdThreads / 32];
    __shared__ __align__(8) uint64_t mbar, cbar;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_abort;

    const SysDev &s = a.s;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int tile = blockIdx.x, e = a.e0 + (int)blockIdx.y;
    unsigned char *ast = a.astage + ((size_t)blockIdx.y * gridDim.x + tile) * a.astage_per;
    const int N = s.n_elec;
    const int spin = e >= s.n_up, ei = spin ? e - s.n_up : e, ns = spin ? s.n_dn : s.n_up;
    const int nspad = a.ns_pad[spin];
    const int mw = a.mw;

    // union of the tile's active shells for electron e, and its AO list
    for (int j = t; j < mw; j += kVdThreads) {
        uint32_t u = 0;
        for (int m = 0; m < TC_M; ++m) {
            const int w = tile * TC_M + m;
            if (w < a.nw) u |= a.masks[((size_t)w * N + e) * mw + j];
        }
        un_s[j] = u;
    }
    __syncthreads();
    const int K = aos_from_mask_n(s, un_s, mw, ao_s, warp_s);
    const int nat = (K + kVdN - 1) / kVdN;
    for (int q = K + t; q < nat * kVdN; q += kVdThreads) ao_s[q] = -1;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;"
                     :: "r"(smem_u32(&tmem_slot)) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar)) : "memory");
        mbar_init(smem_u32(&cbar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t mb = smem_u32(&mbar);
    const uint32_t idesc = umma_idesc_f16_major(TC_M, kVdN, 1, 0, 0);   // BF16, A and B K-major
    const uint64_t kWait = a.wait_ns;
    const uint16_t *Bsl = a.rslice[spin];
    const size_t bstride = (size_t)s.n_ao * nspad;
    const int nst = nspad / kVdK;

    // this CTA's D^-1 rows cut into six exact slices once, for every K stage (the AO tiles
    // reuse them): thread -> (row, chunk of 8 MOs), two per thread
    for (int q = t; q < TC_M * 4; q += kVdThreads) {
        const int prow = q >> 2, pc = q & 3;
        const int pw = tile * TC_M + prow;
        const bool pvalid = pw < a.nw;
        const double *drow = a.Dinv + (size_t)(pvalid ? pw : 0) * a.msz + (spin ? (size_t)s.n_up * s.n_up : 0) +
                             (size_t)ei * ns;
        const int Ep = pvalid ? a.rexp[(size_t)pw * N + e] : 0;
        for (int sg = 0; sg < nst; ++sg) {
            const int k0 = sg * kVdK;
            float sl[8][kC15Slices];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int k = k0 + 8 * pc + i;
                const double d = (pvalid && k < ns) ? drow[k] : 0.0;
                slice6(ff::from_double(d), Ep, sl[i]);
            }
            unsigned char *Ad = ast + (size_t)sg * kC15Slices * kVdPlane;
#pragma unroll
            for (int j = 0; j < kC15Slices; ++j)
                *reinterpret_cast<uint4 *>(Ad + j * kVdPlane + a_off64(prow, pc)) =
                    make_uint4(bf16_pair(sl[0][j], sl[1][j]), bf16_pair(sl[2][j], sl[3][j]),
                               bf16_pair(sl[4][j], sl[5][j]), bf16_pair(sl[6][j], sl[7][j]));
        }
    }
    asm volatile("fence.proxy.async.global;" ::: "memory");   // the staging is read back by bulk copies
    __syncthreads();                                       // the block's global writes, before the copies read them
    const uint32_t cb = smem_u32(&cbar);
    int ncopy = 0;

    // epilogue role: walker row erow (TMEM lane), columns cg * 32 .. + 32 of an AO tile of 64
    const int erow = (warp & 3) * 32 + lane, cg = warp >> 2;
    const int ew = tile * TC_M + erow;
    const bool evalid = ew < a.nw;
    const int Ee = evalid ? a.rexp[(size_t)ew * N + e] : 0;
    const double *rw = a.R + ((size_t)(evalid ? ew : 0) * N + e) * 3;
    const float2 r2[3] = {ff::from_double(rw[0]), ff::from_double(rw[1]), ff::from_double(rw[2])};
    const uint32_t *my_mask = a.masks + ((size_t)(evalid ? ew : 0) * N + e) * mw;
    const uint32_t tlane = (uint32_t)((warp & 3) * 32) << 16;
    // drift and Laplacian accumulated as float pairs on the FP32 pipes (GB300's FP64 rate is 1/64
    // of FP32: FP64 sums here kept the FP64 pipe 30% busy)
    float2 b0 = make_float2(0.f, 0.f), b1 = b0, b2 = b0, lap = b0;

    int ncommit = 0;
    bool ok = true;
    unsigned char *Ab = base;
    unsigned char *Bb = base + kC15Slices * kVdPlane;
    for (int at = 0; at < nat && ok; ++at) {
        for (int sg = 0; sg < nst; ++sg) {
            // the stage buffer: A (the staged D^-1 slices) and B (the rows of A of this AO tile)
            const int k0 = sg * kVdK;
            const unsigned char *As = ast + (size_t)sg * kC15Slices * kVdPlane;
            if (t == 0) {                                  // the staged D^-1 slices: one bulk copy
                mbar_expect_tx(cb, kC15Slices * kVdPlane);
                bulk_g2s(smem_u32(Ab), As, kC15Slices * kVdPlane, cb);
            }
            for (int q = t; q < kC15Slices * kVdN * 4; q += kVdThreads) {
                const int j = q / (kVdN * 4), rem = q - j * (kVdN * 4);
                const int r = rem >> 2, c = rem & 3;
                const int mu = ao_s[at * kVdN + r];
                const bool v = mu >= 0;
                const uint16_t *src = Bsl + j * bstride + (size_t)(v ? mu : 0) * nspad + k0 + 8 * c;
                cp_async16(smem_u32(Bb + j * kVdBPlane + a_off64(r, c)), src, v);
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            ++ncopy;
            // one warp observes the bulk copy (only the MMA issue reads it); the others wait at
            // the barrier without spending issue slots the other CTA's epilogue needs
            if (warp == 0 && !mbar_wait(cb, (ncopy - 1) & 1, kWait)) s_abort = 1;
            __syncthreads();
            if (warp == 0) {                                   // converged: elect.sync per MMA
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint64_t dA = umma_desc_sw64(smem_u32(Ab), 512);
                const uint64_t dB = umma_desc_sw64(smem_u32(Bb), 512);
#pragma unroll
                for (int kk = 0; kk < kVdK / 16; ++kk)
#pragma unroll
                    for (int d = 0; d < kC15Slices; ++d) {
                        const int acc = d < kVdAcc - 1 ? d : kVdAcc - 1;
#pragma unroll
                        for (int i = 0; i <= d; ++i) {
                            const int j = d - i;
                            const uint64_t ad = dA + ((i * kVdPlane + 32 * kk) >> 4);
                            const uint64_t bd = dB + ((j * kVdBPlane + 32 * kk) >> 4);
                            const bool first = sg == 0 && kk == 0 && i == 0 && d <= kVdAcc - 1;
                            umma_bf16_warp(tmem + acc * kVdN, ad, bd, idesc, first ? 0u : 1u);
                        }
                    }
                umma_commit_warp(mb);
            }
            ++ncommit;
            // the buffer is rewritten by the next stage: wait for these MMAs (the other CTA
            // on the SM keeps the tensor pipe busy meanwhile)
            if (warp == 0 && !mbar_wait(mb, (ncommit - 1) & 1, kWait)) s_abort = 1;
            __syncthreads();
            if (s_abort) break;
        }
        ok = !s_abort;
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // epilogue: v for 32 AOs of this walker row, then the AO derivatives at r_e
        FfRadial rd;
        int last_sh = -1;
        float2 *vbuf = reinterpret_cast<float2 *>(base);   // [16][256]: the stage buffer is idle here
        for (int h = 0; h < 2; ++h) {
            const int c0 = cg * 32 + h * 16;
            {
                uint32_t v0[16], v1[16], v2[16], v3[16];
                tmem_ld16(tmem + tlane + (uint32_t)(0 * kVdN + c0), v0);
                tmem_ld16(tmem + tlane + (uint32_t)(1 * kVdN + c0), v1);
                tmem_ld16(tmem + tlane + (uint32_t)(2 * kVdN + c0), v2);
                tmem_ld16(tmem + tlane + (uint32_t)(3 * kVdN + c0), v3);
                // the four order sums (integers in their units) added as a float pair
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    float s, e, s2, e2;
                    ff::two_sum(__uint_as_float(v0[q]), __uint_as_float(v1[q]), s, e);
                    ff::two_sum(s, __uint_as_float(v2[q]), s2, e2);
                    e = __fadd_rn(e, e2);
                    ff::two_sum(s2, __uint_as_float(v3[q]), s, e2);
                    vbuf[q * kVdThreads + t] = ff::renorm(s, __fadd_rn(e, e2));
                }
            }
            if (!evalid) continue;
#pragma unroll 1
            for (int q = 0; q < 16; ++q) {
                const int mu = ao_s[at * kVdN + c0 + q];
                if (mu < 0) break;
                const int sh = s.ao_shell[mu];
                if (!((my_mask[sh >> 5] >> (sh & 31)) & 1u)) continue;
                const int ex = Ee + a.gexp[spin][mu];
                const float2 vr = vbuf[q * kVdThreads + t];
                const float2 vmu = make_float2(scale_pow2(vr.x, ex), scale_pow2(vr.y, ex));   // exact scaling
                if (sh != last_sh) {
                    last_sh = sh;
                    ff_radial(s, a.fb, sh, r2, rd);
                }
                // Laplacian in float-float (the kinetic term cancels against the potential: an FP32
                // Laplacian left E_L at 2e-5 relative on 2048 walkers of 1056 electrons), the
                // gradient in FP32 from the same radial part; products with v and sums in FP64
                float2 val, lp;
                ff_angular(s, a.fb, mu, rd, val, lp);
                const int pw2 = s.ao_pow[mu];
                const int nx = pw2 & 255, ny = (pw2 >> 8) & 255, nz = (pw2 >> 16) & 255;
                const float dx = rd.dx.x + rd.dx.y, dy = rd.dy.x + rd.dy.y, dz = rd.dz.x + rd.dz.y;
                auto ip = [](float x, int n) {
                    float y = 1.f;
                    for (int i = 0; i < n; ++i) y *= x;
                    return y;
                };
                const float px = ip(dx, nx), py = ip(dy, ny), pz = ip(dz, nz);
                const float P = px * py * pz, g = rd.g.x + rd.g.y, m2gd = -2.f * (rd.gd.x + rd.gd.y);
                const float c = a.scf[mu];
                const float g1 = c * ((nx ? nx * ip(dx, nx - 1) : 0.f) * py * pz * g + m2gd * dx * P);
                const float g2 = c * (px * (ny ? ny * ip(dy, ny - 1) : 0.f) * pz * g + m2gd * dy * P);
                const float g3 = c * (px * py * (nz ? nz * ip(dz, nz - 1) : 0.f) * g + m2gd * dz * P);
                b0 = ff::fma2(b0, vmu, make_float2(g1, 0.f));
                b1 = ff::fma2(b1, vmu, make_float2(g2, 0.f));
                b2 = ff::fma2(b2, vmu, make_float2(g3, 0.f));
                lap = ff::fma2(lap, vmu, lp);
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();                                   // TMEM and vbuf read before the next tile
    }
    if (!ok) {
        if (t < TC_M && tile * TC_M + t < a.nw) atomicOr(a.wstatus + tile * TC_M + t, (uint32_t)QMC_STATUS_TIMEOUT);
        asm volatile("cp.async.wait_all;" ::: "memory");
        if (ncopy > 0) mbar_wait(cb, (ncopy - 1) & 1, kDrainNs);        // the last bulk copy
        if (ncommit > 0) mbar_wait(mb, (ncommit - 1) & 1, kDrainNs);   // let MMAs in flight drain
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" :: "r"(tmem) : "memory");
    // the two column groups' partial sums of each row, added in a fixed order
    double *red = reinterpret_cast<double *>(base);        // [2 groups][128 rows][4]; operands no longer read
    red[((size_t)cg * TC_M + erow) * 4 + 0] = ff::val(b0);
    red[((size_t)cg * TC_M + erow) * 4 + 1] = ff::val(b1);
    red[((size_t)cg * TC_M + erow) * 4 + 2] = ff::val(b2);
    red[((size_t)cg * TC_M + erow) * 4 + 3] = ff::val(lap);
    __syncthreads();
    for (int q = t; q < TC_M * 4; q += kVdThreads) {
        const int r = q >> 2, c = q & 3;
        const int w = tile * TC_M + r;
        if (w < a.nw) {
            const double x = red[((size_t)0 * TC_M + r) * 4 + c] + red[((size_t)1 * TC_M + r) * 4 + c];
            a.vd[((size_t)w * N + e) * 4 + c] = ok ? x : __longlong_as_double(0x7ff8000000000000ll);
        }
    }
}

}  // namespace

bool vdrift_fits(const SysDev &s)
{
    const size_t sm = 1024 + (size_t)kVdBuf + sizeof(int) * ((size_t)s.n_ao + kVdN);
    return sm <= 227 * 1024;
}

// electrons per launch (the A staging holds one image per CTA of a batch): up to 264 from 2
// walker tiles on (fewer launches, so fewer partly filled last waves), else up to 64 (one
// walker's scratch stays small); spread evenly over the launches.  Never smaller for more
// tiles, so the staging carved for a walker chunk holds a shorter one's.
int vdrift_batch(const SysDev &s, int tiles)
{
    const int kMax = tiles >= 2 ? 264 : 64;
    if (s.n_elec <= kMax) return s.n_elec;
    const int nl = (s.n_elec + kMax - 1) / kMax;
    return (s.n_elec + nl - 1) / nl;
}

size_t vdrift_stage_per(const SysDev &s)
{
    const int nsmax = s.n_up > s.n_dn ? s.n_up : s.n_dn;
    const size_t nst = (size_t)((nsmax + 63) / 64 * 64) / kVdK;
    return nst * kC15Slices * kVdPlane;
}

size_t vdrift_bytes(const SysDev &s, int nw)
{
    const size_t tiles = (size_t)(nw + TC_M - 1) / TC_M;
    return ((sizeof(int) * (size_t)nw * s.n_elec + 255) / 256) * 256 +
           tiles * (size_t)vdrift_batch(s, (int)tiles) * vdrift_stage_per(s);
}

cudaError_t launch_vdrift(const SysDev &s, const FfBasis &fb, const MixedTables &mt, int nw, const double *R,
                          const uint32_t *masks, int mw, const double *Dinv, double *vd, uint32_t *wstatus,
                          void *scratch, cudaStream_t st, const WaitCfg &wc)
{
    if (nw == 0) return cudaSuccess;
    if (!vdrift_fits(s)) return cudaErrorInvalidConfiguration;
    VdArgs a;
    a.s = s; a.fb = fb; a.R = R; a.masks = masks; a.mw = mw; a.nw = nw; a.Dinv = Dinv;
    a.msz = (size_t)s.n_up * s.n_up + (size_t)s.n_dn * s.n_dn;
    a.rexp = static_cast<const int *>(scratch);
    for (int spin = 0; spin < 2; ++spin) {
        a.rslice[spin] = mt.rslice[spin];
        a.gexp[spin] = mt.gexp[spin];
        a.ns_pad[spin] = mt.ns_pad[spin];
    }
    a.vd = vd;
    a.wstatus = wstatus;
    a.pgf = mt.pgf; a.pcf = mt.pcf; a.scf = mt.scf; a.Qhi = mt.Qhi; a.Qlo = mt.Qlo;
    a.astage = static_cast<unsigned char *>(scratch) + ((sizeof(int) * (size_t)nw * s.n_elec + 255) / 256) * 256;
    a.astage_per = vdrift_stage_per(s);
    a.wait_ns = wc.limit_ns;
    const size_t rows = (size_t)nw * s.n_elec;
    k_vd_rowexp<<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(nw, s.n_up, s.n_dn, a.msz, Dinv,
                                                          static_cast<int *>(scratch));
    const size_t sm = 1024 + (size_t)kVdBuf + sizeof(int) * ((size_t)s.n_ao + kVdN);
    cudaError_t e = cudaFuncSetAttribute(k_vd_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int tiles = (nw + TC_M - 1) / TC_M;
    const int nb = vdrift_batch(s, tiles);
    for (int e0 = 0; e0 < s.n_elec; e0 += nb) {
        a.e0 = e0;
        const int ne = s.n_elec - e0 < nb ? s.n_elec - e0 : nb;
        k_vd_mma<<<dim3(tiles, ne), kVdThreads, sm, st>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace qmc
