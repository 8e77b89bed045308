// Step a7 of the mixed path on the tcgen05 tensor cores:
//
//   dA_s[mu][k] = sum_w g_w sum_{e in s} chi_mu(r_{w,e}) (D^-1)_{w,ek}
//
// (the adjoint of log|Psi| through D_{ke} = sum_mu a_{k mu} chi_mu(r_e) and
// d log|det D| / d D_{ke} = (D^-1)_{ek}, the cofactor identity of Sec. II.C).
//
// It is a contraction over (walker, electron) pairs.  The AOs are grouped into
// blocks of whole atoms (consecutive atoms, at most `nb` AOs: 96, or 64 when a
// spin has more than 640 electrons); a pair is a hit of a block when at least
// one shell of the block is active for it (the exact FP64 screening decisions
// of k_shell_mask).  For one AO block, one spin and wb walkers (8 by default) a CTA forms
//
//   P[k][mu] = sum_{hits h} (D^-1)_{h,k} X[h][mu],   X[h][mu] = g_w chi_mu(r_h)
//
// for all MO tiles of 128 at once: TMEM holds kt * nb FP32 columns (kt = MO
// tiles of the spin), the MO index is the TMEM lane.
//
// Precision.  Both operands are FP32 values split exactly into three BF16
// slices (8 + 8 + 8 significant bits: hi = rn(x), mid = rn(x - hi),
// lo = x - hi - mid, each step exact); the six slice products of order <= 2
// are accumulated in FP32 (the dropped orders are below 2^-22 of a product);
// the accumulation is the dominant error (each MMA rounds the accumulator),
// which is why a CTA sums a few walkers only.
// D^-1 enters rounded to FP32 and chi is evaluated in FP32 (positions as
// float pairs), so a term carries a relative error of a few 2^-24 (up to
// ~1e-6 in the far tail of a Gaussian, where the term itself is ~1e-8 of its
// peak).  Each CTA writes its FP32 partial; the walker blocks' partials are
// summed in FP64.
//
// k_bw_prep:   D^-1 (FP64) -> three BF16 slice planes [w][spin block][e][ns8]
//              (rows padded to a multiple of 8 with zeros), and the electron
//              positions as float pairs.
// k_bw_mma:    per stage of 64 hits: the block's AO values for the hits as
//              three K-major slice planes of X (all threads), and per MO tile
//              the 64 hit rows of the D^-1 slices (cp.async into three MN-major
//              planes, three buffers, one tile ahead); one thread issues the
//              4 x 6 MMAs (M128 N nb K16) of a tile into its accumulator and
//              commits to an mbarrier.  Waits are bounded by %globaltimer; a
//              CTA that gives up writes NaN into its partial.
// k_bw_reduce: dA (+)= sum over walker blocks of the partials, FP64.
#include "qmc_device.cuh"
#include "umma.cuh"

namespace qmc {

constexpr int kBtThreads = 256;
constexpr int kBtHits = 64;                         // hits per stage (K of one stage)
constexpr int kBtScan = 4 * kBtThreads;             // pairs tested per scan round
constexpr int kBtPend = kBtHits + kBtScan;
constexpr int kBtSlices = 3;
constexpr int kBtABufs = 3;
constexpr uint32_t kBtAPlane = kBtHits * TC_N * 2;  // [64 hits][128 MOs] BF16, MN-major: 16 KB
constexpr uint32_t kBtABuf = kBtSlices * kBtAPlane;

struct BwTcArgs {
    SysDev s;
    const float *pgf, *pcf, *scf, *Qhi, *Qlo;
    const float2 *Rf;          // [nw][n_elec][3] positions as float pairs
    const double *g;           // [nw]
    const uint32_t *masks;     // [nw][n_elec][mw]
    int mw;
    const uint16_t *sl;        // [3][nw][msz8] BF16 slices of D^-1
    size_t plane;              // elements of one slice plane (nw * msz8)
    size_t msz8;               // padded elements per walker
    size_t soff8[2];           // first element of the spin block within a walker
    int ns8[2];                // padded row length per spin
    int nw;                    // walkers of this chunk
    int wb;                    // walkers per CTA
    int nb;                    // AO block width = TMEM columns per MO tile
    const int *blk_ao0, *blk_sh0;
    float *part[2];            // [walker block][n_ao][ns] FP32 partials
    unsigned long long wait_ns;  // limit of each wait (WaitCfg)
    int expire_w;              // test hook: spin-up CTAs of this walker (in the pass) let their last wait run out
};

__device__ __forceinline__ float ipowf(float x, int n)
{
    float y = 1.f;
    for (int i = 0; i < n; ++i) y *= x;
    return y;
}

// any shell in [sh0, sh1) active in the mask words mk
__device__ __forceinline__ bool block_hit(const uint32_t *mk, int sh0, int sh1)
{
    const int w0 = sh0 >> 5, w1 = (sh1 - 1) >> 5;
    uint32_t any = 0;
    for (int wd = w0; wd <= w1; ++wd) {
        uint32_t m = mk[wd];
        if (wd == w0) m &= 0xffffffffu << (sh0 & 31);
        if (wd == w1) m &= 0xffffffffu >> (31 - ((sh1 - 1) & 31));
        any |= m;
    }
    return any != 0u;
}

// x = hi + mid + lo exactly (x FP32, each part BF16)
__device__ __forceinline__ void slice3(float x, __nv_bfloat16 &b0, __nv_bfloat16 &b1, __nv_bfloat16 &b2)
{
    b0 = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(b0);
    b1 = __float2bfloat16_rn(r1);
    b2 = __float2bfloat16_rn(r1 - __bfloat162float(b1));
}

__global__ void k_bw_prep(const double *__restrict__ dinv, int nw, int n_up, int n_dn, int ns8u, int ns8d,
                          size_t msz8, uint16_t *__restrict__ sl, size_t plane, const double *__restrict__ R,
                          int n_elec, float2 *__restrict__ Rf)
{
    const size_t msz = (size_t)n_up * n_up + (size_t)n_dn * n_dn;
    const size_t up8 = (size_t)n_up * ns8u;
    const size_t per = msz8 / 8;
    const size_t nchunk = (size_t)nw * per;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nchunk; q += stride) {
        const size_t w = q / per;
        size_t r = (q - w * per) * 8;
        const int spin = r >= up8;
        if (spin) r -= up8;
        const int ns = spin ? n_dn : n_up, ns8 = spin ? ns8d : ns8u;
        const int e = (int)(r / ns8), k = (int)(r - (size_t)e * ns8);
        const double *src = dinv + w * msz + (spin ? (size_t)n_up * n_up : 0) + (size_t)e * ns;
        uint32_t o[kBtSlices][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float x0 = k + 2 * i < ns ? (float)src[k + 2 * i] : 0.f;
            const float x1 = k + 2 * i + 1 < ns ? (float)src[k + 2 * i + 1] : 0.f;
            __nv_bfloat16 a[3], b[3];
            slice3(x0, a[0], a[1], a[2]);
            slice3(x1, b[0], b[1], b[2]);
#pragma unroll
            for (int p = 0; p < kBtSlices; ++p) {
                __nv_bfloat162 v;
                v.x = a[p];
                v.y = b[p];
                o[p][i] = *reinterpret_cast<const uint32_t *>(&v);
            }
        }
        const size_t dst = w * msz8 + (spin ? up8 : 0) + (size_t)e * ns8 + k;
#pragma unroll
        for (int p = 0; p < kBtSlices; ++p)
            *reinterpret_cast<uint4 *>(sl + p * plane + dst) = make_uint4(o[p][0], o[p][1], o[p][2], o[p][3]);
    }
    const size_t npos = (size_t)nw * n_elec * 3;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < npos; q += stride) {
        const double v = R[q];
        const float h = (float)v;
        Rf[q] = make_float2(h, (float)(v - (double)h));
    }
}

__global__ void __launch_bounds__(kBtThreads, 1) k_bw_mma(BwTcArgs a)
{
    extern __shared__ __align__(1024) unsigned char bt_smem[];
    unsigned char *base = bt_smem + ((1024 - (smem_u32(bt_smem) & 1023)) & 1023);
    const uint32_t xplane = (uint32_t)a.nb * 128;            // [nb rows][64 hits] BF16, K-major
    unsigned char *abuf = base;                               // kBtABufs x [3 planes]
    unsigned char *xbuf = base + kBtABufs * kBtABuf;          // 2 stages x [3 planes]
    __shared__ int hits_s[2][kBtHits];                        // (walker in block) << 16 | electron in spin
    __shared__ int pend_s[kBtPend];
    __shared__ int warp_s[kBtThreads / 32];
    __shared__ __align__(8) uint64_t mbar[kBtABufs];
    __shared__ uint32_t tmem_slot;
    __shared__ int s_npend, s_abort, s_never;

    const SysDev &s = a.s;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int blk = blockIdx.x, spin = blockIdx.y, wblk = blockIdx.z;
    const int ns = spin ? s.n_dn : s.n_up;
    if (ns == 0) return;
    const int e0 = spin ? s.n_up : 0;
    const int kts = (ns + TC_N - 1) / TC_N;
    const int ao0 = a.blk_ao0[blk], nao = a.blk_ao0[blk + 1] - ao0;
    const int sh0 = a.blk_sh0[blk], sh1 = a.blk_sh0[blk + 1];
    const int w_lo = wblk * a.wb;
    const int nwl = min(a.wb, a.nw - w_lo);
    const int npairs = nwl * ns;
    float *part = a.part[spin] + (size_t)wblk * s.n_ao * ns;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;"
                     :: "r"(smem_u32(&tmem_slot)) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        for (int b = 0; b < kBtABufs; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar[b])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_npend = 0;
        s_abort = 0;
        s_never = 0;
    }
    // rows nb..: never written again; rows < nao are rewritten every stage
    for (uint32_t q = t; q < 2 * kBtSlices * xplane / 16; q += kBtThreads)
        reinterpret_cast<uint4 *>(xbuf)[q] = make_uint4(0u, 0u, 0u, 0u);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    uint32_t mbs[kBtABufs];
    for (int b = 0; b < kBtABufs; ++b) mbs[b] = smem_u32(&mbar[b]);
    const uint64_t kWait = a.wait_ns;
    const bool expire = spin == 0 && a.expire_w >= w_lo && a.expire_w < w_lo + nwl;
    const uint32_t idesc = umma_idesc_f16_major(TC_M, a.nb, 1, 1, 0);   // A = D^-1 rows MN-major, B = X K-major

    // next stage of up to 64 hits into hits_s[buf]; returns their number
    int scan_pos = 0;
    auto next_stage = [&](int buf) -> int {
        while (s_npend < kBtHits && scan_pos < npairs) {
            int code[4], hit[4], cnt = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int p = scan_pos + i * kBtThreads + t;
                hit[i] = 0;
                code[i] = 0;
                if (p < npairs) {
                    const int wl = p / ns, e = p - wl * ns;
                    const int w = w_lo + wl;
                    if (a.g[w] != 0.0) {
                        const uint32_t *mk = a.masks + ((size_t)w * s.n_elec + e0 + e) * a.mw;
                        hit[i] = block_hit(mk, sh0, sh1);
                    }
                    code[i] = (wl << 16) | e;
                }
                cnt += hit[i];
            }
            const int base_n = s_npend;
            int total;
            int o = base_n + block_excl_scan<kBtThreads>(cnt, warp_s, &total);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (hit[i]) pend_s[o++] = code[i];
            __syncthreads();
            if (t == 0) s_npend = base_n + total;
            scan_pos += kBtScan;
            __syncthreads();
        }
        const int np = s_npend, n = min(np, kBtHits);
        if (t < n) hits_s[buf][t] = pend_s[t];
        int keep[kBtPend / kBtThreads + 1];
#pragma unroll
        for (int i = 0; i < kBtPend / kBtThreads + 1; ++i) {
            const int q = t + i * kBtThreads;
            keep[i] = q < np - n ? pend_s[n + q] : 0;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kBtPend / kBtThreads + 1; ++i) {
            const int q = t + i * kBtThreads;
            if (q < np - n) pend_s[q] = keep[i];
        }
        if (t == 0) s_npend = np - n;
        __syncthreads();
        return n;
    };

    // X slice planes of stage buffer sb: four threads per hit, shells of the block split four ways
    auto produce_x = [&](int sb, int nh) {
        unsigned char *xb = xbuf + (size_t)sb * kBtSlices * xplane;
        const int h = t & (kBtHits - 1), q = t >> 6;
        const bool valid = h < nh;
        const int code = valid ? hits_s[sb][h] : 0;
        const int w = w_lo + (code >> 16), e = code & 0xffff;
        const size_t pe = (size_t)w * s.n_elec + e0 + e;
        const uint32_t *mk = a.masks + pe * a.mw;
        float2 rx = make_float2(0.f, 0.f), ry = rx, rz = rx;
        float gw = 0.f;
        if (valid) {
            rx = a.Rf[3 * pe];
            ry = a.Rf[3 * pe + 1];
            rz = a.Rf[3 * pe + 2];
            gw = (float)a.g[w];
        }
        for (int sh = sh0 + q; sh < sh1; sh += kBtThreads / kBtHits) {
            const int r0 = s.sh_ao0[sh] - ao0, nc = ncart(s.sh_L[sh]);
            const bool act = valid && ((mk[sh >> 5] >> (sh & 31)) & 1u);
            float dx = 0.f, dy = 0.f, dz = 0.f, gr = 0.f;
            if (act) {
                const int at = s.sh_atom[sh];
                dx = (rx.x - a.Qhi[3 * at]) + (rx.y - a.Qlo[3 * at]);
                dy = (ry.x - a.Qhi[3 * at + 1]) + (ry.y - a.Qlo[3 * at + 1]);
                dz = (rz.x - a.Qhi[3 * at + 2]) + (rz.y - a.Qlo[3 * at + 2]);
                const float d2 = dx * dx + dy * dy + dz * dz;
                const int p0 = s.sh_pstart[sh], np = s.sh_nprim[sh];
                for (int p = 0; p < np; ++p) gr += a.pcf[p0 + p] * expf(-a.pgf[p0 + p] * d2);
                gr *= gw;
            }
            for (int c = 0; c < nc; ++c) {
                float x = 0.f;
                if (act) {
                    const int mu = ao0 + r0 + c;
                    const int pw = s.ao_pow[mu];
                    x = a.scf[mu] * (ipowf(dx, pw & 255) * ipowf(dy, (pw >> 8) & 255) * ipowf(dz, (pw >> 16) & 255)) *
                        gr;
                }
                __nv_bfloat16 b0, b1, b2;
                slice3(x, b0, b1, b2);
                const uint32_t off = a_off(r0 + c, h >> 3) + (uint32_t)(h & 7) * 2;
                *reinterpret_cast<__nv_bfloat16 *>(xb + off) = b0;
                *reinterpret_cast<__nv_bfloat16 *>(xb + xplane + off) = b1;
                *reinterpret_cast<__nv_bfloat16 *>(xb + 2 * xplane + off) = b2;
            }
        }
    };

    // cp.async of MO tile `tile` of the D^-1 slice rows of the hits of stage buffer sb into A buffer ab
    auto issue_a = [&](int sb, int nh, int tile, int ab) {
        unsigned char *A = abuf + (size_t)ab * kBtABuf;
        const int k0 = tile * TC_N;
        const int ns8 = a.ns8[spin];
        for (int q = t; q < kBtSlices * kBtHits * (TC_N / 8); q += kBtThreads) {
            const int p = q / (kBtHits * (TC_N / 8)), rem = q - p * (kBtHits * (TC_N / 8));
            const int h = rem / (TC_N / 8), c = rem - h * (TC_N / 8);
            const bool v = h < nh && k0 + 8 * c < ns8;
            const uint16_t *src = a.sl;
            if (v) {
                const int code = hits_s[sb][h];
                const int w = w_lo + (code >> 16), e = code & 0xffff;
                src = a.sl + p * a.plane + (size_t)w * a.msz8 + a.soff8[spin] + (size_t)e * ns8 + k0 + 8 * c;
            }
            cp_async16(smem_u32(A + p * kBtAPlane + b_off(h, 8 * c)), src, v);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };

    // the 4 x 6 MMAs of one (stage, MO tile) step
    auto mma = [&](int sb, int tile, int ab, bool first) {
        const uint32_t a0 = smem_u32(abuf + (size_t)ab * kBtABuf);
        const uint32_t x0 = smem_u32(xbuf + (size_t)sb * kBtSlices * xplane);
        const uint64_t dA = umma_desc(a0, kBLbo, kBSbo);
        const uint64_t dX = umma_desc(x0, 16, 1024);
        const uint32_t d = tmem + (uint32_t)(tile * a.nb);
#pragma unroll
        for (int kk = 0; kk < kBtHits / 16; ++kk)
#pragma unroll
            for (int ord = 0; ord < kBtSlices; ++ord)
#pragma unroll
                for (int i = 0; i <= ord; ++i) {
                    const int j = ord - i;
                    const uint64_t ad = dA + ((i * kBtAPlane + 2 * kk * kBSbo) >> 4);
                    const uint64_t xd = dX + ((j * xplane + 32 * kk) >> 4);
                    umma_bf16_warp(d, ad, xd, idesc, (first && kk == 0 && ord == 0) ? 0u : 1u);
                }
    };

    int nh[2] = {0, 0};
    int ncommit = 0;
    bool ok = true;
    nh[0] = next_stage(0);
    if (nh[0] > 0) {
        issue_a(0, nh[0], 0, 0);
        produce_x(0, nh[0]);
        int j = 0, stage = 0, tile = 0;
        while (true) {
            // prepare step j + 1 while the MMAs of step j - 1 run
            int tn = tile + 1, sn = stage;
            if (tn == kts) {
                tn = 0;
                sn = stage + 1;
            }
            const int jn = j + 1;
            bool has_next = true;
            if (tn == 0) {
                nh[sn & 1] = next_stage(sn & 1);
                has_next = nh[sn & 1] > 0;
            }
            if (has_next) {
                // A buffer jn % 3 was read by step jn - 3; the X buffer of stage sn by stage sn - 2,
                // whose last step is jn - 1 - kts (covered by jn - 3 unless kts == 1)
                const int need = (tn == 0 && kts == 1) ? jn - 2 : jn - 3;
                if (need >= 0 && !mbar_wait(mbs[need % kBtABufs], (need / kBtABufs) & 1, kWait)) s_abort = 1;
                issue_a(sn & 1, nh[sn & 1], tn, jn % kBtABufs);
                if (tn == 0) produce_x(sn & 1, nh[sn & 1]);
                asm volatile("cp.async.wait_group 1;" ::: "memory");
            } else {
                asm volatile("cp.async.wait_group 0;" ::: "memory");
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (s_abort) {
                ok = false;
                break;
            }
            if (warp == 0) {                              // converged: elect.sync per MMA
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                mma(stage & 1, tile, j % kBtABufs, stage == 0);
                umma_commit_warp(mbs[j % kBtABufs]);
            }
            ncommit = j + 1;
            if (!has_next) break;
            j = jn;
            tile = tn;
            stage = sn;
        }
        if (ok) {
            const int last = ncommit - 1;
            if (expire ? !flag_wait(&s_never, kWait) : !mbar_wait(mbs[last % kBtABufs], (last / kBtABufs) & 1, kWait))
                s_abort = 1;
        }
        __syncthreads();
        ok = ok && !s_abort;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int quad = warp & 3;
    for (int tile = 0; tile < kts; ++tile)
        for (int cb = (warp >> 2) * 32; cb < a.nb; cb += 64) {
            uint32_t v[32];
            if (ncommit > 0 && ok) tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(tile * a.nb + cb), v);
            const int k = tile * TC_N + quad * 32 + lane;
            if (k < ns) {
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    if (cb + q >= nao) break;
                    const float val = !ok ? __int_as_float(0x7fc00000) : (ncommit > 0 ? __uint_as_float(v[q]) : 0.f);
                    part[(size_t)(ao0 + cb + q) * ns + k] = val;
                }
            }
        }
    if (!ok) {
        asm volatile("cp.async.wait_all;" ::: "memory");
        for (int b = 0; b < kBtABufs; ++b) {   // let MMAs in flight drain before TMEM is released
            const int x = ncommit - 1 - (((ncommit - 1 - b) % kBtABufs) + kBtABufs) % kBtABufs;
            if (x >= 0) mbar_wait(mbs[b], (x / kBtABufs) & 1, kDrainNs);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" :: "r"(tmem) : "memory");
}

__global__ void k_bw_reduce(const float *__restrict__ part, int nwb, size_t n, double *__restrict__ dA, int accumulate)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += stride) {
        double acc = accumulate ? dA[q] : 0.0;
        for (int b = 0; b < nwb; ++b) acc += (double)part[(size_t)b * n + q];
        dA[q] = acc;
    }
}

namespace {
size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
int round8(int n) { return (n + 7) & ~7; }
size_t msz8_of(const SysDev &s) { return (size_t)s.n_up * round8(s.n_up) + (size_t)s.n_dn * round8(s.n_dn); }

size_t chunk_bytes(const SysDev &s, int mw, int wc, int wb)
{
    const size_t nwb = (size_t)(wc + wb - 1) / wb;
    return al256((size_t)wc * s.n_elec * mw * 4) + al256((size_t)kBtSlices * wc * msz8_of(s) * 2) +
           al256((size_t)wc * s.n_elec * 3 * sizeof(float2)) + al256(nwb * s.n_ao * (size_t)s.n_elec * 4);
}

size_t smem_bytes(int nb) { return 1024 + kBtABufs * (size_t)kBtABuf + 2 * (size_t)kBtSlices * nb * 128; }
}  // namespace

int bwtc_block_width(int nmax)
{
    const int kt = (nmax + TC_N - 1) / TC_N;
    return kt <= 5 ? 96 : (kt <= 8 ? 64 : 0);
}

size_t bwtc_bytes(const SysDev &s, int mw, int nw, int wb)
{
    const int wc = nw < 1 ? 1 : (nw > kBwtChunk ? kBwtChunk : nw);
    return chunk_bytes(s, mw, wc, wb);
}

cudaError_t launch_backward_tc(const SysDev &s, const MixedTables &mt, const BwBlocks &bb, int wb, int nw,
                               const double *R, const double *dinv, const double *g, double *dA_up, double *dA_dn, void *ws,
                               size_t ws_bytes, cudaStream_t st, const WaitCfg &wcfg)
{
    cudaError_t e;
    if (nw == 0) {
        if ((e = cudaMemsetAsync(dA_up, 0, sizeof(double) * s.n_ao * (size_t)s.n_up, st)) != cudaSuccess) return e;
        return cudaMemsetAsync(dA_dn, 0, sizeof(double) * s.n_ao * (size_t)s.n_dn, st);
    }
    const int mw = mt.mask_words;
    // walkers per pass: whole walker blocks, as many as the workspace holds
    if (wb < 1) return cudaErrorInvalidValue;
    int wc = nw < kBwtChunk ? nw : kBwtChunk;
    while (wc > wb && chunk_bytes(s, mw, wc, wb) > ws_bytes) wc = ((wc - 1) / wb) * wb;
    while (wc > 1 && chunk_bytes(s, mw, wc, wb) > ws_bytes) wc /= 2;
    if (chunk_bytes(s, mw, wc, wb) > ws_bytes) return cudaErrorMemoryAllocation;
    const size_t sm = smem_bytes(bb.nb);
    if (sm > 227 * 1024) return cudaErrorInvalidConfiguration;
    if ((e = cudaFuncSetAttribute(k_bw_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess)
        return e;

    const int ns8u = round8(s.n_up), ns8d = round8(s.n_dn);
    const size_t msz8 = msz8_of(s), msz = (size_t)s.n_up * s.n_up + (size_t)s.n_dn * s.n_dn;
    const size_t nwb_max = (size_t)(wc + wb - 1) / wb;
    char *p = static_cast<char *>(ws);
    uint32_t *masks = reinterpret_cast<uint32_t *>(p);
    p += al256((size_t)wc * s.n_elec * mw * 4);
    uint16_t *sl = reinterpret_cast<uint16_t *>(p);
    p += al256((size_t)kBtSlices * wc * msz8 * 2);
    float2 *Rf = reinterpret_cast<float2 *>(p);
    p += al256((size_t)wc * s.n_elec * 3 * sizeof(float2));
    float *part = reinterpret_cast<float *>(p);

    BwTcArgs a;
    a.s = s;
    a.pgf = mt.pgf; a.pcf = mt.pcf; a.scf = mt.scf; a.Qhi = mt.Qhi; a.Qlo = mt.Qlo;
    a.Rf = Rf;
    a.masks = masks;
    a.mw = mw;
    a.sl = sl;
    a.msz8 = msz8;
    a.soff8[0] = 0;
    a.soff8[1] = (size_t)s.n_up * ns8u;
    a.ns8[0] = ns8u;
    a.ns8[1] = ns8d;
    a.nb = bb.nb;
    a.wb = wb;
    a.blk_ao0 = bb.ao0;
    a.blk_sh0 = bb.sh0;
    a.part[0] = part;
    a.part[1] = part + nwb_max * s.n_ao * (size_t)s.n_up;
    for (int c0 = 0; c0 < nw; c0 += wc) {
        const int n = nw - c0 < wc ? nw - c0 : wc;
        const int nwb = (n + wb - 1) / wb;
        const double *Rc = R + (size_t)c0 * s.n_elec * 3;
        if ((e = launch_shell_mask(s, mt, n, Rc, mw, masks, st)) != cudaSuccess) return e;
        a.plane = (size_t)n * msz8;
        a.nw = n;
        a.g = g + c0;
        a.wait_ns = wcfg.limit_ns;
        a.expire_w = (wcfg.expire_kernels & QMC_EXPIRE_ADJOINT) && wcfg.expire_w >= c0 && wcfg.expire_w < c0 + n
                         ? wcfg.expire_w - c0 : -1;
        const size_t work = (size_t)n * (msz8 / 8);
        const int pblocks = (int)((work + 255) / 256 < 152 * 16 ? (work + 255) / 256 : 152 * 16);
        k_bw_prep<<<pblocks, 256, 0, st>>>(dinv + (size_t)c0 * msz, n, s.n_up, s.n_dn, ns8u, ns8d, msz8, sl, a.plane,
                                           Rc, s.n_elec, Rf);
        k_bw_mma<<<dim3(bb.nblk, 2, nwb), kBtThreads, sm, st>>>(a);
        for (int spin = 0; spin < 2; ++spin) {
            const size_t cnt = (size_t)s.n_ao * (spin ? s.n_dn : s.n_up);
            if (cnt == 0) continue;
            const int rblocks = (int)((cnt + 255) / 256 < 152 * 8 ? (cnt + 255) / 256 : 152 * 8);
            k_bw_reduce<<<rblocks, 256, 0, st>>>(a.part[spin], nwb, cnt, spin ? dA_dn : dA_up, c0 > 0);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace qmc
