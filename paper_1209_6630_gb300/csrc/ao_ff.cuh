// Float-float AO values and Laplacians, and the union AO list of a CTA's
// walkers, shared by the mixed path's C1/C5 kernels.
#pragma once

#include "ff_math.cuh"
#include "qmc_device.cuh"

namespace qmc {

__device__ __forceinline__ float2 ff_ipow(float2 x, int n)   // x^n, n <= 4
{
    switch (n) {
    case 0: return make_float2(1.f, 0.f);
    case 1: return x;
    case 2: return ff::mul(x, x);
    case 3: return ff::mul(ff::mul(x, x), x);
    case 4: { const float2 y = ff::mul(x, x); return ff::mul(y, y); }
    default: return make_float2(0.f, 0.f);
    }
}

// Value and Laplacian of AO mu (the two quantities C1 and C5 need) at the
// position r (three float pairs), in float-float arithmetic:
//   chi = c P(d) g(d2),  g = sum_p c_p e^{-gamma_p d2},  P = dx^nx dy^ny dz^nz
//   lap chi = c (lap P g + P (gl - 4 L gd)),  gd = sum_p c_p gamma_p e_p,
//                                            gl = sum_p c_p (4 gamma_p d2 - 6) gamma_p e_p
// (the FP64 formulas of the other paths, each operation on float pairs).
// The radial part (d, g, gd, gl) is shared by the AOs of a shell.
struct FfRadial {
    float2 dx, dy, dz, g, gd, gl;
};

__device__ __forceinline__ void ff_radial(const SysDev &s, const FfBasis &fb, int sh, const float2 *r, FfRadial &o)
{
    const int a = s.sh_atom[sh];
    o.dx = ff::sub(r[0], fb.Q[3 * a]);
    o.dy = ff::sub(r[1], fb.Q[3 * a + 1]);
    o.dz = ff::sub(r[2], fb.Q[3 * a + 2]);
    const float2 d2 = ff::add(ff::add(ff::mul(o.dx, o.dx), ff::mul(o.dy, o.dy)), ff::mul(o.dz, o.dz));
    float2 g = make_float2(0.f, 0.f), gd = g, gl = g;
    const int p0 = s.sh_pstart[sh], np = s.sh_nprim[sh];
    for (int p = 0; p < np; ++p) {
        const float2 gam = fb.pg[p0 + p];
        const float2 x = ff::mul(gam, d2);
        const float2 ce = ff::mul(fb.pc[p0 + p], ff::exp_neg(x, fb.expj));
        g = ff::add(g, ce);
        const float2 gce = ff::mul(gam, ce);
        gd = ff::add(gd, gce);
        const float2 t = ff::add(make_float2(4.f * x.x, 4.f * x.y), make_float2(-6.f, 0.f));
        gl = ff::fma2(gl, t, gce);
    }
    o.g = g;
    o.gd = gd;
    o.gl = gl;
}

__device__ __forceinline__ void ff_angular(const SysDev &s, const FfBasis &fb, int mu, const FfRadial &rd,
                                           float2 &val, float2 &lap)
{
    const int pw = s.ao_pow[mu];
    const int nx = pw & 255, ny = (pw >> 8) & 255, nz = (pw >> 16) & 255;
    const int L = nx + ny + nz;
    const float2 c = fb.sc[mu];
    if (L == 0) {
        val = ff::mul(c, rd.g);
        lap = ff::mul(c, rd.gl);
        return;
    }
    const float2 px = ff_ipow(rd.dx, nx), py = ff_ipow(rd.dy, ny), pz = ff_ipow(rd.dz, nz);
    const float2 pyz = ff::mul(py, pz);
    const float2 P = ff::mul(px, pyz);
    float2 lapP = make_float2(0.f, 0.f);
    if (nx > 1) lapP = ff::mulf(ff::mul(ff_ipow(rd.dx, nx - 2), pyz), (float)(nx * (nx - 1)));
    if (ny > 1)
        lapP = ff::add(lapP, ff::mulf(ff::mul(ff::mul(px, ff_ipow(rd.dy, ny - 2)), pz), (float)(ny * (ny - 1))));
    if (nz > 1)
        lapP = ff::add(lapP, ff::mulf(ff::mul(ff::mul(px, py), ff_ipow(rd.dz, nz - 2)), (float)(nz * (nz - 1))));
    val = ff::mul(c, ff::mul(P, rd.g));
    const float2 inner = ff::fma2(ff::mul(lapP, rd.g), P, ff::sub(rd.gl, ff::mulf(rd.gd, (float)(4 * L))));
    lap = ff::mul(c, inner);
}

__device__ __forceinline__ void ao_val_lap_ff(const SysDev &s, const FfBasis &fb, int mu, const float2 *r,
                                              float2 &val, float2 &lap)
{
    FfRadial rd;
    ff_radial(s, fb, s.ao_shell[mu], r, rd);
    ff_angular(s, fb, mu, rd, val, lap);
}

// Value alone (the C-free variant's C1): the radial sum g without gd and gl.
__device__ __forceinline__ float2 ao_val_ff(const SysDev &s, const FfBasis &fb, int mu, const float2 *r)
{
    const int sh = s.ao_shell[mu];
    const int a = s.sh_atom[sh];
    const float2 dx = ff::sub(r[0], fb.Q[3 * a]), dy = ff::sub(r[1], fb.Q[3 * a + 1]), dz = ff::sub(r[2], fb.Q[3 * a + 2]);
    const float2 d2 = ff::add(ff::add(ff::mul(dx, dx), ff::mul(dy, dy)), ff::mul(dz, dz));
    float2 g = make_float2(0.f, 0.f);
    const int p0 = s.sh_pstart[sh], np = s.sh_nprim[sh];
    for (int p = 0; p < np; ++p)
        g = ff::add(g, ff::mul(fb.pc[p0 + p], ff::exp_neg(ff::mul(fb.pg[p0 + p], d2), fb.expj)));
    const int pw = s.ao_pow[mu];
    const int nx = pw & 255, ny = (pw >> 8) & 255, nz = (pw >> 16) & 255;
    const float2 P = ff::mul(ff_ipow(dx, nx), ff::mul(ff_ipow(dy, ny), ff_ipow(dz, nz)));
    return ff::mul(fb.sc[mu], ff::mul(P, g));
}

// Ordered list of the AOs of the shells set in `bits` for a block of any
// size (a multiple of 32 threads).  Returns the count; idx_s receives the AO indices.
static __device__ int aos_from_mask_n(const SysDev &s, const uint32_t *bits, int mw, int *idx_s, int *warp_s)
{
    const int nthr = blockDim.x, nwarps = nthr >> 5, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int words_per = (mw + nthr - 1) / nthr;
    const int w0 = min((int)threadIdx.x * words_per, mw), w1 = min(w0 + words_per, mw);
    int nao = 0;
    for (int j = w0; j < w1; ++j)
        for (uint32_t b = bits[j]; b; b &= b - 1) nao += ncart(s.sh_L[j * 32 + __ffs(b) - 1]);
    // exclusive block scan of nao
    int x = nao;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_s[wid] = x;
    __syncthreads();
    int base = 0, total = 0;
    for (int q = 0; q < nwarps; ++q) {
        const int v = warp_s[q];
        if (q < wid) base += v;
        total += v;
    }
    __syncthreads();
    int off = base + x - nao;
    for (int j = w0; j < w1; ++j)
        for (uint32_t b = bits[j]; b; b &= b - 1) {
            const int sh = j * 32 + __ffs(b) - 1;
            const int a0 = s.sh_ao0[sh], nc = ncart(s.sh_L[sh]);
            for (int c = 0; c < nc; ++c, ++off) idx_s[off] = a0 + c;
        }
    __syncthreads();
    return total;
}

}  // namespace qmc
