// Host side of libqmcgb: system loading, workspace planning and the C ABI
// entry points declared in include/qmcgb.h.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include "qmc_internal.cuh"

namespace qmc {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

int cuda_fail(cudaError_t e, const char *where)
{
    set_error(std::string(where) + ": " + cudaGetErrorString(e));
    return QMC_ERR_CUDA;
}

static int invalid(const std::string &msg)
{
    set_error(msg);
    return QMC_ERR_INVALID;
}

static int ncart_h(int L) { return (L + 1) * (L + 2) / 2; }

// CRC-32 of ISO 3309 / ITU-T V.42 (reflected polynomial 0xEDB88320), the key
// the paper attaches to a simulation's critical data (Sec. V.C).  crc32_update
// advances the register over `n` bytes (table built from the polynomial on
// first use); a key is crc32_update(0xFFFFFFFF, ...) ^ 0xFFFFFFFF.
static uint32_t crc32_update(uint32_t reg, const void *data, size_t n)
{
    static uint32_t table[256];
    static std::once_flag once;
    std::call_once(once, [] {
        for (uint32_t i = 0; i < 256; ++i) {
            uint32_t c = i;
            for (int k = 0; k < 8; ++k) c = (c & 1u) ? (0xEDB88320u ^ (c >> 1)) : (c >> 1);
            table[i] = c;
        }
    });
    const unsigned char *p = static_cast<const unsigned char *>(data);
    for (size_t i = 0; i < n; ++i) reg = table[(reg ^ p[i]) & 0xFFu] ^ (reg >> 8);
    return reg;
}

// Register after the basis part of a description (Z .. ao_scale).
static uint32_t desc_crc_prefix(const qmc_system_desc *d)
{
    uint32_t r = 0xFFFFFFFFu;
    r = crc32_update(r, d->Z, sizeof(double) * (size_t)d->n_atom);
    r = crc32_update(r, d->Q, sizeof(double) * 3 * (size_t)d->n_atom);
    r = crc32_update(r, d->shell_atom, sizeof(int32_t) * (size_t)d->n_shell);
    r = crc32_update(r, d->shell_L, sizeof(int32_t) * (size_t)d->n_shell);
    r = crc32_update(r, d->shell_nprim, sizeof(int32_t) * (size_t)d->n_shell);
    r = crc32_update(r, d->shell_pstart, sizeof(int32_t) * (size_t)d->n_shell);
    r = crc32_update(r, d->prim_gamma, sizeof(double) * (size_t)d->n_prim);
    r = crc32_update(r, d->prim_coef, sizeof(double) * (size_t)d->n_prim);
    r = crc32_update(r, d->ao_shell, sizeof(int32_t) * (size_t)d->n_ao);
    r = crc32_update(r, d->ao_pow, sizeof(int32_t) * 3 * (size_t)d->n_ao);
    r = crc32_update(r, d->ao_scale, sizeof(double) * (size_t)d->n_ao);
    return r;
}

// Key from the prefix register, the MO coefficients and eps.
static uint32_t desc_crc_finish(uint32_t r, int nao, int nu, int nd, int a_dtype, const void *A_up, const void *A_dn,
                                double eps)
{
    const size_t es = a_dtype == QMC_DTYPE_F64 ? 8 : 4;
    if (nu) r = crc32_update(r, A_up, es * (size_t)nao * nu);
    if (nd) r = crc32_update(r, A_dn, es * (size_t)nao * nd);
    r = crc32_update(r, &eps, sizeof(double));
    return r ^ 0xFFFFFFFFu;
}

// Radial part of shell sh at squared distance x: sum_p c_p exp(-gamma_p x),
// summed in primitive order (the same operations on every call).
static double shell_radial(const qmc_system_desc *d, int sh, double x)
{
    double g = 0.0;
    const int p0 = d->shell_pstart[sh];
    for (int p = 0; p < d->shell_nprim[sh]; ++p) g = g + d->prim_coef[p0 + p] * exp(-d->prim_gamma[p0 + p] * x);
    return g;
}

// Screening radius of a shell (Sec. III): the smallest non-negative double x
// with g(x) < eps.  Non-negative doubles are ordered like their bit patterns,
// so bisection on the 64-bit patterns between a point with g >= eps and a
// point with g < eps ends on two neighbouring doubles.
static double shell_radius2(const qmc_system_desc *d, int sh)
{
    const double eps = d->eps;
    if (shell_radial(d, sh, 0.0) < eps) return 0.0;
    double hi = 1.0;
    while (!(shell_radial(d, sh, hi) < eps)) hi = hi * 2.0;
    long long lo_bits, hi_bits;
    double zero = 0.0;
    memcpy(&lo_bits, &zero, 8);
    memcpy(&hi_bits, &hi, 8);
    while (hi_bits - lo_bits > 1) {
        const long long mid = lo_bits + (hi_bits - lo_bits) / 2;
        double xm;
        memcpy(&xm, &mid, 8);
        if (shell_radial(d, sh, xm) < eps) hi_bits = mid; else lo_bits = mid;
    }
    double r2;
    memcpy(&r2, &hi_bits, 8);
    return r2;
}

// float -> bfloat16 bits, round to nearest even
static uint16_t bf16_bits(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

static float bf16_value(uint16_t b)
{
    const uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

// Upper bounds of |d chi / dx_l| (out[0]) and |lap chi| (out[1]) over the
// screened sphere d2 < R2 of a shell, from |x|,|y|,|z| <= r on a radial grid
// (with a 25% margin); used to pick exact power-of-two scales for FP16.
static void shell_deriv_bound(const qmc_system_desc *d, int sh, int ao0, double R2, double out[2])
{
    const int L = d->shell_L[sh], p0 = d->shell_pstart[sh], np = d->shell_nprim[sh];
    double sc = 0.0;
    for (int c = 0; c < ncart_h(L); ++c) sc = std::max(sc, fabs(d->ao_scale[ao0 + c]));
    const double rmax = sqrt(std::max(R2, 0.0));
    double bg = 0.0, bl = 0.0;
    const int npt = 4096;
    for (int i = 0; i <= npt; ++i) {
        const double r = rmax * i / npt, r2 = r * r;
        double G = 0.0, GD = 0.0, GL = 0.0;
        for (int q = 0; q < np; ++q) {
            const double gam = d->prim_gamma[p0 + q], c = fabs(d->prim_coef[p0 + q]), ex = exp(-gam * r2);
            G += c * ex;
            GD += c * gam * ex;
            GL += c * fabs(4.0 * gam * gam * r2 - 6.0 * gam) * ex;
        }
        const double rL = pow(r, L), rL1 = L >= 1 ? pow(r, L - 1) : 0.0, rL2 = L >= 2 ? pow(r, L - 2) : 0.0;
        bg = std::max(bg, sc * (L * rL1 * G + 2.0 * r * rL * GD));
        bl = std::max(bl, sc * (L * (L - 1) * rL2 * G + rL * (GL + 4.0 * L * GD)));
    }
    out[0] = 1.25 * bg;
    out[1] = 1.25 * bl;
}

struct Blob {
    std::vector<char> host;
    size_t add(const void *src, size_t bytes)
    {
        const size_t off = (host.size() + 255) & ~size_t(255);
        host.resize(off + bytes);
        if (bytes) memcpy(host.data() + off, src, bytes);
        return off;
    }
};

// Device copies of the MO coefficients: FP64 [n_ao][n_s]; BF16 hi/lo planes
// and FP16 hi/lo planes of A * 2^a_exp, [n_ao][n_s padded to 64]; float-float
// planes [n_ao][n_s].  a_exp is chosen so that max |A| * 2^a_exp <= 8192.
struct MoLayout {
    size_t oA[2], oBh[2], oBl[2], oHh[2], oHl[2], oF[2], oCm[2], oSl[2], oFe[2], oRs[2], oGe[2];
    int ns_pad[2], ns32[2], a_exp[2];
};

static void build_mo(int nao, int nu, int nd, int a_dtype, const void *A_up, const void *A_dn, Blob &b,
                     MoLayout &L)
{
    for (int spin = 0; spin < 2; ++spin) {
        const int ns = spin ? nd : nu;
        const void *src = spin ? A_dn : A_up;
        std::vector<double> A64((size_t)nao * ns);
        for (size_t q = 0; q < A64.size(); ++q)
            A64[q] = a_dtype == QMC_DTYPE_F64 ? static_cast<const double *>(src)[q]
                                              : (double) static_cast<const float *>(src)[q];
        L.oA[spin] = b.add(A64.data(), sizeof(double) * A64.size());
        const int np = ((ns + 63) / 64) * 64;
        L.ns_pad[spin] = np;
        double amax = 0.0;
        for (double a : A64) amax = std::max(amax, fabs(a));
        L.a_exp[spin] = amax > 0.0 ? (int)floor(log2(8192.0 / amax)) : 0;
        const double asc = ldexp(1.0, L.a_exp[spin]);
        std::vector<uint16_t> bh((size_t)nao * np, 0), bl((size_t)nao * np, 0);
        std::vector<uint16_t> hh((size_t)nao * np, 0), hl((size_t)nao * np, 0);
        const int n32 = ((ns + 31) / 32) * 32;
        L.ns32[spin] = n32;
        std::vector<float2> ff((size_t)nao * n32, float2{0.f, 0.f});
        for (int mu = 0; mu < nao; ++mu)
            for (int k = 0; k < ns; ++k) {
                const double a = A64[(size_t)mu * ns + k];
                const uint16_t h = bf16_bits((float)a);
                bh[(size_t)mu * np + k] = h;
                bl[(size_t)mu * np + k] = bf16_bits((float)(a - (double)bf16_value(h)));
                const double as = a * asc;
                const __half h16 = __float2half_rn((float)as);
                const __half l16 = __float2half_rn((float)(as - (double)__half2float(h16)));
                memcpy(&hh[(size_t)mu * np + k], &h16, 2);
                memcpy(&hl[(size_t)mu * np + k], &l16, 2);
                const float f = (float)a;
                ff[(size_t)mu * n32 + k] = float2{f, (float)(a - (double)f)};
            }
        L.oBh[spin] = b.add(bh.data(), 2 * bh.size());
        L.oBl[spin] = b.add(bl.data(), 2 * bl.size());
        L.oHh[spin] = b.add(hh.data(), 2 * hh.size());
        L.oHl[spin] = b.add(hl.data(), 2 * hl.size());
        L.oF[spin] = b.add(ff.data(), sizeof(float2) * ff.size());
        std::vector<float> cm(n32, 0.0f);
        for (int mu = 0; mu < nao; ++mu)
            for (int k = 0; k < ns; ++k) cm[k] = std::max(cm[k], (float)fabs(A64[(size_t)mu * ns + k]));
        L.oCm[spin] = b.add(cm.data(), 4 * cm.size());
        // exact BF16 slices of A[mu][k] 2^-F_k, F_k = the column's exponent bound
        std::vector<int> fe(np, 0);
        for (int k = 0; k < ns; ++k) {
            double m = 0.0;
            for (int mu = 0; mu < nao; ++mu) m = std::max(m, fabs(A64[(size_t)mu * ns + k]));
            fe[k] = m > 0.0 ? ilogb(m) + 1 : 0;
        }
        std::vector<uint16_t> sl((size_t)kC15Slices * nao * np, 0);
        for (int mu = 0; mu < nao; ++mu)
            for (int k = 0; k < ns; ++k) {
                double r = ldexp(A64[(size_t)mu * ns + k], -fe[k]);
                for (int j = 0; j < kC15Slices; ++j) {
                    const int sh = kC15SliceBits * (j + 1);
                    const double sj = ldexp(nearbyint(ldexp(r, sh)), -sh);
                    sl[((size_t)j * nao + mu) * np + k] = bf16_bits((float)sj);
                    r -= sj;
                }
            }
        L.oSl[spin] = b.add(sl.data(), 2 * sl.size());
        L.oFe[spin] = b.add(fe.data(), 4 * fe.size());
        // the same slicing with one exponent per AO row: the operand of v = D^-1 A^T, whose
        // contraction runs over the MO index k
        std::vector<int> ge(nao, 0);
        for (int mu = 0; mu < nao; ++mu) {
            double m = 0.0;
            for (int k = 0; k < ns; ++k) m = std::max(m, fabs(A64[(size_t)mu * ns + k]));
            ge[mu] = m > 0.0 ? ilogb(m) + 1 : 0;
        }
        std::vector<uint16_t> rs((size_t)kC15Slices * nao * np, 0);
        for (int mu = 0; mu < nao; ++mu)
            for (int k = 0; k < ns; ++k) {
                double r = ldexp(A64[(size_t)mu * ns + k], -ge[mu]);
                for (int j = 0; j < kC15Slices; ++j) {
                    const int sh = kC15SliceBits * (j + 1);
                    const double sj = ldexp(nearbyint(ldexp(r, sh)), -sh);
                    rs[((size_t)j * nao + mu) * np + k] = bf16_bits((float)sj);
                    r -= sj;
                }
            }
        L.oRs[spin] = b.add(rs.data(), 2 * rs.size());
        L.oGe[spin] = b.add(ge.data(), 4 * ge.size());
    }
}

static void point_mo(qmc_system *sys, char *dev, const MoLayout &L)
{
    MixedTables &mt = sys->mixed;
    for (int spin = 0; spin < 2; ++spin) {
        sys->d.A64[spin] = reinterpret_cast<const double *>(dev + L.oA[spin]);
        mt.bhi[spin] = reinterpret_cast<const uint16_t *>(dev + L.oBh[spin]);
        mt.blo[spin] = reinterpret_cast<const uint16_t *>(dev + L.oBl[spin]);
        mt.hhi[spin] = reinterpret_cast<const uint16_t *>(dev + L.oHh[spin]);
        mt.hlo[spin] = reinterpret_cast<const uint16_t *>(dev + L.oHl[spin]);
        mt.ff[spin] = reinterpret_cast<const float2 *>(dev + L.oF[spin]);
        mt.ns32[spin] = L.ns32[spin];
        mt.colmax[spin] = reinterpret_cast<const float *>(dev + L.oCm[spin]);
        mt.slice[spin] = reinterpret_cast<const uint16_t *>(dev + L.oSl[spin]);
        mt.fexp[spin] = reinterpret_cast<const int *>(dev + L.oFe[spin]);
        mt.rslice[spin] = reinterpret_cast<const uint16_t *>(dev + L.oRs[spin]);
        mt.gexp[spin] = reinterpret_cast<const int *>(dev + L.oGe[spin]);
        mt.ns_pad[spin] = L.ns_pad[spin];
        mt.a_exp[spin] = L.a_exp[spin];
    }
}

}  // namespace qmc

using namespace qmc;

extern "C" const char *qmc_last_error(void) { return g_err.c_str(); }

extern "C" const char *qmc_version(void) { return "qmcgb 0.1 (sm_103a)"; }

extern "C" int qmc_system_load(const qmc_system_desc *d, int device, qmc_system **out)
{
    if (!d || !out) return invalid("qmc_system_load: null argument");
    *out = nullptr;
    if (d->n_atom <= 0 || d->n_shell <= 0 || d->n_ao <= 0 || d->n_prim <= 0)
        return invalid("qmc_system_load: empty system");
    if (d->n_up < 0 || d->n_dn < 0 || d->n_up + d->n_dn == 0)
        return invalid("qmc_system_load: electron counts");
    if (d->n_up > kMaxN || d->n_dn > kMaxN) return invalid("qmc_system_load: more than 1024 electrons of one spin");
    if (d->n_shell > 64 * 128) return invalid("qmc_system_load: more than 8192 shells");
    if (!(d->eps > 0.0)) return invalid("qmc_system_load: eps must be > 0");
    if (d->a_dtype != QMC_DTYPE_F64 && d->a_dtype != QMC_DTYPE_F32) return invalid("qmc_system_load: a_dtype");
    if (!d->Z || !d->Q || !d->shell_atom || !d->shell_L || !d->shell_nprim || !d->shell_pstart || !d->prim_gamma ||
        !d->prim_coef || !d->ao_shell || !d->ao_pow || !d->ao_scale || (d->n_up && !d->A_up) || (d->n_dn && !d->A_dn))
        return invalid("qmc_system_load: null array");
    // Sec. V.C: the CRC-32 key checks that the critical data arrived intact
    const uint32_t crc_pre = desc_crc_prefix(d);
    const uint32_t crc = desc_crc_finish(crc_pre, d->n_ao, d->n_up, d->n_dn, d->a_dtype, d->A_up, d->A_dn, d->eps);
    if (crc != d->crc32) {
        char msg[160];
        snprintf(msg, sizeof msg, "qmc_system_load: CRC-32 of the description is 0x%08x, desc->crc32 is 0x%08x",
                 crc, d->crc32);
        return invalid(msg);
    }

    const int na = d->n_atom, nsh = d->n_shell, nao = d->n_ao, nu = d->n_up, nd = d->n_dn;
    std::vector<int> atom_sh0(na + 1, 0), sh_ao0(nsh, -1);
    for (int s = 0; s < nsh; ++s) {
        const int a = d->shell_atom[s];
        if (a < 0 || a >= na || (s > 0 && a < d->shell_atom[s - 1]))
            return invalid("qmc_system_load: shells must be sorted by atom");
        if (d->shell_L[s] < 0 || d->shell_L[s] > kMaxL) return invalid("qmc_system_load: shell L outside 0..4");
        if (d->shell_nprim[s] < 1 || d->shell_nprim[s] > kMaxPrim) return invalid("qmc_system_load: 1..16 primitives");
        if (d->shell_pstart[s] < 0 || d->shell_pstart[s] + d->shell_nprim[s] > d->n_prim)
            return invalid("qmc_system_load: primitive range");
        for (int p = 0; p < d->shell_nprim[s]; ++p)
            if (!(d->prim_gamma[d->shell_pstart[s] + p] > 0.0)) return invalid("qmc_system_load: exponent <= 0");
        atom_sh0[a + 1] += 1;
    }
    for (int a = 0; a < na; ++a) atom_sh0[a + 1] += atom_sh0[a];
    int max_ao_atom = 0;
    {
        int mu = 0;
        for (int s = 0; s < nsh; ++s) {
            sh_ao0[s] = mu;
            const int L = d->shell_L[s];
            for (int c = 0; c < ncart_h(L); ++c, ++mu) {
                if (mu >= nao || d->ao_shell[mu] != s) return invalid("qmc_system_load: AOs must be stored shell by shell");
                const int *pw = d->ao_pow + 3 * mu;
                if (pw[0] < 0 || pw[1] < 0 || pw[2] < 0 || pw[0] + pw[1] + pw[2] != L)
                    return invalid("qmc_system_load: AO powers must sum to L");
            }
        }
        if (mu != nao) return invalid("qmc_system_load: n_ao does not match the shells");
        for (int a = 0; a < na; ++a) {
            if (atom_sh0[a + 1] == atom_sh0[a]) continue;
            const int last = atom_sh0[a + 1] - 1;
            max_ao_atom = std::max(max_ao_atom, sh_ao0[last] + ncart_h(d->shell_L[last]) - sh_ao0[atom_sh0[a]]);
        }
        if (max_ao_atom > 32) return invalid("qmc_system_load: more than 32 AOs on one atom");
    }

    qmc_system *sys = new qmc_system();
    sys->device = device;
    sys->crc_prefix = crc_pre;
    sys->crc = crc;
    sys->crc_nojas = crc;
    sys->eps = d->eps;
    sys->tiles.wait_s = 2.0;
    sys->tiles.expire_walker = -1;
    sys->tiles.expire_kernels = QMC_EXPIRE_C15 | QMC_EXPIRE_A4 | QMC_EXPIRE_ADJOINT;
    sys->tiles.gj_panel = (d->n_up > 640 || d->n_dn > 640) ? 8 : 16;
    sys->tiles.c15_walkers = 4;
    // the tensor-core panel updates win from ~500 electrons per spin on (measured at 434 / 528 / 866)
    sys->tiles.a4_mode = (std::max(nu, nd) >= 512 && gjtc_fits(std::max(nu, nd))) ? QMC_A4_TENSOR : QMC_A4_FLOAT_FLOAT;
    // kappa_inf overstates the 2-norm condition by up to ~n: small matrices need a lower bar
    // (158 electrons x 4096 walkers: 1e8 left one walker at |dlog|Psi|| = 1.4e-6, 1e7 at most
    // 6e-8 for 7% more a4 time); their FP64 recomputation is cheap
    sys->tiles.a4_kappa_max = std::max(nu, nd) <= 256 ? 1e7 : 1e8;
    // the FP64 path's 1e-10 bar on E_L: measured on 512 walkers of 1056 electrons, kappa_inf
    // 1e6 keeps every walker within 4.2e-11 (1e7: 12 walkers above 1e-10); at 158 electrons the
    // float-pair elimination alone moved one walker's E_L by 1.3e-10 (kappa_inf below 1e3, T
    // and V cancelling), so small systems recompute every matrix in FP64
    sys->tiles.f64_kappa_max = std::max(nu, nd) <= 256 ? 1.0 : 1e6;
    sys->max_shell_per_atom = max_ao_atom;
    sys->R2_host.resize(nsh);
    std::vector<double> atom_R2(na, 0.0);
    for (int s = 0; s < nsh; ++s) {
        sys->R2_host[s] = shell_radius2(d, s);
        atom_R2[d->shell_atom[s]] = std::max(atom_R2[d->shell_atom[s]], sys->R2_host[s]);
    }
    double vnn = 0.0;
    for (int a = 0; a < na; ++a)
        for (int b = a + 1; b < na; ++b) {
            const double dx = d->Q[3 * a] - d->Q[3 * b], dy = d->Q[3 * a + 1] - d->Q[3 * b + 1],
                         dz = d->Q[3 * a + 2] - d->Q[3 * b + 2];
            vnn += d->Z[a] * d->Z[b] / sqrt(dx * dx + dy * dy + dz * dz);
        }

    std::vector<int> ao_pow(nao);
    for (int mu = 0; mu < nao; ++mu)
        ao_pow[mu] = d->ao_pow[3 * mu] | (d->ao_pow[3 * mu + 1] << 8) | (d->ao_pow[3 * mu + 2] << 16);
    Blob b;
    const size_t oQ = b.add(d->Q, sizeof(double) * 3 * na);
    const size_t oZ = b.add(d->Z, sizeof(double) * na);
    const size_t oAS = b.add(atom_sh0.data(), sizeof(int) * (na + 1));
    const size_t oAR = b.add(atom_R2.data(), sizeof(double) * na);
    const size_t oSA = b.add(d->shell_atom, sizeof(int) * nsh);
    const size_t oSL = b.add(d->shell_L, sizeof(int) * nsh);
    const size_t oSN = b.add(d->shell_nprim, sizeof(int) * nsh);
    const size_t oSP = b.add(d->shell_pstart, sizeof(int) * nsh);
    const size_t oSO = b.add(sh_ao0.data(), sizeof(int) * nsh);
    const size_t oSR = b.add(sys->R2_host.data(), sizeof(double) * nsh);
    const size_t oPG = b.add(d->prim_gamma, sizeof(double) * d->n_prim);
    const size_t oPC = b.add(d->prim_coef, sizeof(double) * d->n_prim);
    const size_t oAP = b.add(ao_pow.data(), sizeof(int) * nao);
    const size_t oAO = b.add(d->ao_shell, sizeof(int) * nao);
    const size_t oSC = b.add(d->ao_scale, sizeof(double) * nao);
    // FP32 copies of the basis tables and float-pair positions for the tensor-core producer
    std::vector<float> pgf(d->n_prim), pcf(d->n_prim), scf(nao), qhi(3 * na), qlo(3 * na);
    for (int q = 0; q < d->n_prim; ++q) { pgf[q] = (float)d->prim_gamma[q]; pcf[q] = (float)d->prim_coef[q]; }
    for (int mu = 0; mu < nao; ++mu) scf[mu] = (float)d->ao_scale[mu];
    for (int q = 0; q < 3 * na; ++q) { qhi[q] = (float)d->Q[q]; qlo[q] = (float)(d->Q[q] - (double)qhi[q]); }
    const size_t oPgf = b.add(pgf.data(), 4 * pgf.size()), oPcf = b.add(pcf.data(), 4 * pcf.size());
    const size_t oScf = b.add(scf.data(), 4 * scf.size());
    const size_t oQh = b.add(qhi.data(), 4 * qhi.size()), oQl = b.add(qlo.data(), 4 * qlo.size());
    // float-pair tables for the float-float AO evaluation of C1/C5
    auto pair = [](double v) { const float h = (float)v; return float2{h, (float)(v - (double)h)}; };
    std::vector<float2> pg2(d->n_prim), pc2(d->n_prim), sc2(nao), q2(3 * na), ej(25);
    for (int q = 0; q < d->n_prim; ++q) { pg2[q] = pair(d->prim_gamma[q]); pc2[q] = pair(d->prim_coef[q]); }
    for (int mu = 0; mu < nao; ++mu) sc2[mu] = pair(d->ao_scale[mu]);
    for (int q = 0; q < 3 * na; ++q) q2[q] = pair(d->Q[q]);
    for (int j = -12; j <= 12; ++j) ej[j + 12] = pair(exp(-j / 32.0));
    const size_t oPg2 = b.add(pg2.data(), 8 * pg2.size()), oPc2 = b.add(pc2.data(), 8 * pc2.size());
    const size_t oSc2 = b.add(sc2.data(), 8 * sc2.size()), oQ2 = b.add(q2.data(), 8 * q2.size());
    const size_t oEj = b.add(ej.data(), 8 * ej.size());
    std::vector<float> ar2f(na), sr2f(nsh);
    for (int a = 0; a < na; ++a) ar2f[a] = (float)atom_R2[a];
    for (int sh = 0; sh < nsh; ++sh) sr2f[sh] = (float)sys->R2_host[sh];
    const size_t oAR2f = b.add(ar2f.data(), 4 * ar2f.size()), oSR2f = b.add(sr2f.data(), 4 * sr2f.size());
    // AO blocks of the tensor-core adjoint: consecutive atoms, at most nb AOs per block
    const int nb_bw = bwtc_block_width(std::max(nu, nd));
    std::vector<int> bw_ao0, bw_sh0;
    {
        int cnt = 0;
        for (int a = 0; a < na; ++a) {
            const int s0 = atom_sh0[a], s1 = atom_sh0[a + 1];
            if (s1 == s0) continue;
            const int n_a = sh_ao0[s1 - 1] + ncart_h(d->shell_L[s1 - 1]) - sh_ao0[s0];
            if (bw_ao0.empty() || cnt + n_a > nb_bw) {
                bw_ao0.push_back(sh_ao0[s0]);
                bw_sh0.push_back(s0);
                cnt = 0;
            }
            cnt += n_a;
        }
        bw_ao0.push_back(nao);
        bw_sh0.push_back(nsh);
    }
    const size_t oBA = b.add(bw_ao0.data(), 4 * bw_ao0.size()), oBS = b.add(bw_sh0.data(), 4 * bw_sh0.size());
    // Jastrow e-n parameters (set by qmc_system_set_jastrow; off at load)
    std::vector<double> jzero(na, 0.0);
    const size_t oJa = b.add(jzero.data(), 8 * jzero.size()), oJb = b.add(jzero.data(), 8 * jzero.size());
    // AO derivative values enter the FP16 split scaled by 2^b_exp (bound * 2^b_exp <= 8192)
    double dbound[2] = {0.0, 0.0};
    for (int sh = 0; sh < nsh; ++sh) {
        double bd[2];
        shell_deriv_bound(d, sh, sh_ao0[sh], sys->R2_host[sh], bd);
        dbound[0] = std::max(dbound[0], bd[0]);
        dbound[1] = std::max(dbound[1], bd[1]);
    }
    const int b_exp = dbound[0] > 0.0 ? std::min(24, (int)floor(log2(8192.0 / dbound[0]))) : 0;

    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) { delete sys; return cuda_fail(e, "qmc_system_load: cudaSetDevice"); }
    char *dev = nullptr;
    e = cudaMalloc(&dev, b.host.size());
    if (e != cudaSuccess) { delete sys; return cuda_fail(e, "qmc_system_load: cudaMalloc"); }
    sys->allocs.push_back(dev);
    e = cudaMemcpy(dev, b.host.data(), b.host.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { qmc_system_free(sys); return cuda_fail(e, "qmc_system_load: cudaMemcpy"); }
    Blob bm;
    MoLayout mo;
    build_mo(nao, nu, nd, d->a_dtype, d->A_up, d->A_dn, bm, mo);
    char *mdev = nullptr;
    e = cudaMalloc(&mdev, bm.host.size());
    if (e != cudaSuccess) { qmc_system_free(sys); return cuda_fail(e, "qmc_system_load: cudaMalloc"); }
    sys->allocs.push_back(mdev);
    e = cudaMemcpy(mdev, bm.host.data(), bm.host.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { qmc_system_free(sys); return cuda_fail(e, "qmc_system_load: cudaMemcpy"); }
    sys->mo_dev = mdev;
    sys->mo_bytes = bm.host.size();
    sys->a_dtype = d->a_dtype;
    point_mo(sys, mdev, mo);

    SysDev &s = sys->d;
    s.n_atom = na; s.n_shell = nsh; s.n_ao = nao; s.n_up = nu; s.n_dn = nd; s.n_elec = nu + nd;
    s.Q = reinterpret_cast<const double *>(dev + oQ);
    s.Z = reinterpret_cast<const double *>(dev + oZ);
    s.atom_sh0 = reinterpret_cast<const int *>(dev + oAS);
    s.atom_R2 = reinterpret_cast<const double *>(dev + oAR);
    s.sh_atom = reinterpret_cast<const int *>(dev + oSA);
    s.sh_L = reinterpret_cast<const int *>(dev + oSL);
    s.sh_nprim = reinterpret_cast<const int *>(dev + oSN);
    s.sh_pstart = reinterpret_cast<const int *>(dev + oSP);
    s.sh_ao0 = reinterpret_cast<const int *>(dev + oSO);
    s.sh_R2 = reinterpret_cast<const double *>(dev + oSR);
    s.pg = reinterpret_cast<const double *>(dev + oPG);
    s.pc = reinterpret_cast<const double *>(dev + oPC);
    s.ao_pow = reinterpret_cast<const int *>(dev + oAP);
    s.ao_shell = reinterpret_cast<const int *>(dev + oAO);
    s.ao_scale = reinterpret_cast<const double *>(dev + oSC);
    s.vnn = vnn;
    s.jas = 0;
    s.ja_par = s.ja_anti = s.jb_ee = 0.0;
    s.ja_en = reinterpret_cast<const double *>(dev + oJa);
    s.jb_en = reinterpret_cast<const double *>(dev + oJb);
    MixedTables &mt = sys->mixed;
    mt.b_exp = b_exp;
    mt.mask_words = (nsh + 31) / 32;
    mt.pgf = reinterpret_cast<const float *>(dev + oPgf);
    mt.pcf = reinterpret_cast<const float *>(dev + oPcf);
    mt.scf = reinterpret_cast<const float *>(dev + oScf);
    mt.Qhi = reinterpret_cast<const float *>(dev + oQh);
    mt.Qlo = reinterpret_cast<const float *>(dev + oQl);
    // the C-free variant where its kernels fit (1056 electrons x 2048 walkers: 468 against 545 ms
    // per step, drift 6e-7 normwise against 1e-4), else C1..C5 on the tensor cores, else float-float
    sys->tiles.c15_mode = !c15tc_fits(s, mt.mask_words) ? QMC_C15_FLOAT_FLOAT
                          : (vdrift_fits(s) ? QMC_C15_CFREE : QMC_C15_TENSOR);
    sys->tiles.bw_walkers = 8;
    sys->bw.nblk = (int)bw_ao0.size() - 1;
    sys->bw.nb = nb_bw;
    sys->bw.ao0 = reinterpret_cast<const int *>(dev + oBA);
    sys->bw.sh0 = reinterpret_cast<const int *>(dev + oBS);
    mt.atom_R2f = reinterpret_cast<const float *>(dev + oAR2f);
    mt.sh_R2f = reinterpret_cast<const float *>(dev + oSR2f);
    mt.ffb.pg = reinterpret_cast<const float2 *>(dev + oPg2);
    mt.ffb.pc = reinterpret_cast<const float2 *>(dev + oPc2);
    mt.ffb.sc = reinterpret_cast<const float2 *>(dev + oSc2);
    mt.ffb.Q = reinterpret_cast<const float2 *>(dev + oQ2);
    mt.ffb.expj = reinterpret_cast<const float2 *>(dev + oEj);
    *out = sys;
    return QMC_OK;
}

extern "C" int qmc_system_set_mo(qmc_system *sys, int a_dtype, const void *A_up, const void *A_dn)
{
    if (!sys) return invalid("qmc_system_set_mo: null system");
    if (a_dtype != QMC_DTYPE_F64 && a_dtype != QMC_DTYPE_F32) return invalid("qmc_system_set_mo: a_dtype");
    if ((sys->d.n_up && !A_up) || (sys->d.n_dn && !A_dn)) return invalid("qmc_system_set_mo: null matrix");
    Blob bm;
    MoLayout mo;
    build_mo(sys->d.n_ao, sys->d.n_up, sys->d.n_dn, a_dtype, A_up, A_dn, bm, mo);
    if (bm.host.size() != sys->mo_bytes) return invalid("qmc_system_set_mo: layout mismatch");
    cudaError_t e = cudaSetDevice(sys->device);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();   // no evaluation may still read the old tables
    if (e == cudaSuccess) e = cudaMemcpy(sys->mo_dev, bm.host.data(), bm.host.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "qmc_system_set_mo");
    sys->a_dtype = a_dtype;
    point_mo(sys, static_cast<char *>(sys->mo_dev), mo);
    sys->crc = desc_crc_finish(sys->crc_prefix, sys->d.n_ao, sys->d.n_up, sys->d.n_dn, a_dtype, A_up, A_dn, sys->eps);
    sys->crc_nojas = sys->crc;
    sys->d.jas = 0;          // new coefficients: a Jastrow factor must be set again (and keyed again)
    return QMC_OK;
}

extern "C" int qmc_system_set_jastrow(qmc_system *sys, const qmc_jastrow *j)
{
    if (!sys) return invalid("qmc_system_set_jastrow: null system");
    const int na = sys->d.n_atom;
    if (!j || !j->enabled) {
        sys->d.jas = 0;
        sys->crc = sys->crc_nojas;
        return QMC_OK;
    }
    if (!j->a_en || !j->b_en) return invalid("qmc_system_set_jastrow: null e-n parameters");
    const double sc[3] = {j->a_par, j->a_anti, j->b_ee};
    for (double x : sc)
        if (!isfinite(x)) return invalid("qmc_system_set_jastrow: non-finite parameter");
    if (j->b_ee < 0.0) return invalid("qmc_system_set_jastrow: b_ee must be >= 0");
    for (int a = 0; a < na; ++a)
        if (!isfinite(j->a_en[a]) || !(j->b_en[a] >= 0.0))
            return invalid("qmc_system_set_jastrow: e-n parameters must be finite with b_en >= 0");
    cudaError_t e = cudaSetDevice(sys->device);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();   // no evaluation may still read the old values
    if (e == cudaSuccess)
        e = cudaMemcpy(const_cast<double *>(sys->d.ja_en), j->a_en, sizeof(double) * na, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(const_cast<double *>(sys->d.jb_en), j->b_en, sizeof(double) * na, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "qmc_system_set_jastrow");
    sys->d.jas = 1;
    sys->d.ja_par = j->a_par;
    sys->d.ja_anti = j->a_anti;
    sys->d.jb_ee = j->b_ee;
    // the Jastrow parameters are critical data too (Sec. V.C): the key continues over them
    uint32_t r = sys->crc_nojas ^ 0xFFFFFFFFu;
    r = crc32_update(r, sc, sizeof sc);
    r = crc32_update(r, j->a_en, sizeof(double) * na);
    r = crc32_update(r, j->b_en, sizeof(double) * na);
    sys->crc = r ^ 0xFFFFFFFFu;
    return QMC_OK;
}

extern "C" int qmc_system_crc32(const qmc_system *sys, uint32_t *crc)
{
    if (!sys || !crc) return invalid("qmc_system_crc32: null argument");
    *crc = sys->crc;
    return QMC_OK;
}

extern "C" int qmc_system_set_tiles(qmc_system *sys, const qmc_tiles *tiles)
{
    if (!sys || !tiles) return invalid("qmc_system_set_tiles: null argument");
    if (tiles->gj_panel != 8 && tiles->gj_panel != 16 && tiles->gj_panel != 32)
        return invalid("qmc_system_set_tiles: gj_panel must be 8, 16 or 32");
    if (tiles->c15_walkers != 2 && tiles->c15_walkers != 4)
        return invalid("qmc_system_set_tiles: c15_walkers must be 2 or 4");
    if (tiles->a4_mode != QMC_A4_FP64 && tiles->a4_mode != QMC_A4_FLOAT_FLOAT && tiles->a4_mode != QMC_A4_TENSOR)
        return invalid("qmc_system_set_tiles: a4_mode");
    if (tiles->a4_mode == QMC_A4_TENSOR && !gjtc_fits(std::max(sys->d.n_up, sys->d.n_dn)))
        return invalid("qmc_system_set_tiles: a4_mode tensor exceeds the panel kernel's shared memory");
    if (tiles->c15_mode != QMC_C15_FLOAT_FLOAT && tiles->c15_mode != QMC_C15_TENSOR && tiles->c15_mode != QMC_C15_CFREE)
        return invalid("qmc_system_set_tiles: c15_mode");
    if ((tiles->c15_mode == QMC_C15_TENSOR || tiles->c15_mode == QMC_C15_CFREE) &&
        !c15tc_fits(sys->d, sys->mixed.mask_words))
        return invalid("qmc_system_set_tiles: c15_mode tensor exceeds the kernel's shared-memory limits");
    if (tiles->c15_mode == QMC_C15_CFREE && !vdrift_fits(sys->d))
        return invalid("qmc_system_set_tiles: c15_mode cfree exceeds the drift kernel's shared-memory limits");
    if (!(tiles->a4_kappa_max > 0.0)) return invalid("qmc_system_set_tiles: a4_kappa_max must be > 0");
    if (!(tiles->f64_kappa_max > 0.0)) return invalid("qmc_system_set_tiles: f64_kappa_max must be > 0");
    if (tiles->bw_walkers != 2 && tiles->bw_walkers != 4 && tiles->bw_walkers != 8 && tiles->bw_walkers != 16 &&
        tiles->bw_walkers != 32)
        return invalid("qmc_system_set_tiles: bw_walkers must be 2, 4, 8, 16 or 32");
    if (!(tiles->wait_s >= 1e-6 && tiles->wait_s <= 60.0))
        return invalid("qmc_system_set_tiles: wait_s must be within 1e-6 .. 60 seconds");
    if (tiles->expire_walker < -1) return invalid("qmc_system_set_tiles: expire_walker must be >= -1");
    if (tiles->expire_kernels < 0 || tiles->expire_kernels > 7)
        return invalid("qmc_system_set_tiles: expire_kernels must be a combination of QMC_EXPIRE_* bits");
    sys->tiles = *tiles;
    return QMC_OK;
}

extern "C" int qmc_system_get_tiles(const qmc_system *sys, qmc_tiles *tiles)
{
    if (!sys || !tiles) return invalid("qmc_system_get_tiles: null argument");
    *tiles = sys->tiles;
    return QMC_OK;
}

extern "C" int qmc_system_free(qmc_system *sys)
{
    if (!sys) return QMC_OK;
    int rc = QMC_OK;
    for (void *p : sys->allocs)
        if (p) {
            cudaError_t e = cudaFree(p);
            if (e != cudaSuccess) rc = cuda_fail(e, "qmc_system_free: cudaFree");
        }
    delete sys;
    return rc;
}

extern "C" int qmc_system_shell_r2(const qmc_system *sys, double *R2_host)
{
    if (!sys || !R2_host) return invalid("qmc_system_shell_r2: null argument");
    memcpy(R2_host, sys->R2_host.data(), sizeof(double) * sys->R2_host.size());
    return QMC_OK;
}

// ---------------------------------------------------------------------------
// Workspace plan per walker: X (C1 in FP64, LU input), Cd (C2..C5), Dinv,
// per-spin log|det| and sign, status bits.
cudaError_t qmc::tmap_encode(CUtensorMap *m, CUtensorMapDataType dt, int rank, const void *addr,
                             const uint64_t *dims, const uint64_t *strides, const uint32_t *box,
                             CUtensorMapSwizzle swz)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    static std::once_flag once;
    static cudaError_t init_err = cudaSuccess;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult qr;
        init_err = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &qr);
        if (init_err == cudaSuccess && (qr != cudaDriverEntryPointSuccess || !f)) init_err = cudaErrorSymbolNotFound;
        if (init_err == cudaSuccess) encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    });
    if (init_err != cudaSuccess) return init_err;
    if (rank < 1 || rank > 5) return cudaErrorInvalidValue;
    cuuint64_t d[5], st[4];
    cuuint32_t b[5], es[5];
    for (int i = 0; i < rank; ++i) {
        d[i] = dims[i];
        b[i] = box[i];
        es[i] = 1;
        if (i > 0) st[i - 1] = strides[i - 1];
    }
    memset(m, 0, sizeof(CUtensorMap));
    const CUresult r = encode(m, dt, (cuuint32_t)rank, const_cast<void *>(addr), d, st, b, es,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

namespace {

struct Plan {
    size_t msz;        // n_up^2 + n_dn^2
    size_t per_walker; // bytes
    bool mixed;
    bool ffgj;         // a4 on float pairs (+ FP64 recompute flags)
    bool tcgj;         // ... with the panel updates on the tensor cores (scratch per chunk)
    size_t cd_bytes;   // per walker: FP64 path C2..C5 in FP64; mixed C2..C4 FP32 + C5 FP64
    size_t mask_bytes; // per walker (mixed path): N x mask_words x 4
    size_t redo_bytes; // per chunk (float-float a4): list and state of the FP64 recomputation
    bool c15tc;        // C1/C5 on the tensor cores (staging buffer per chunk)
    bool cfree;        // C-free variant: C1 alone, drift and Laplacian from v = D^-1 A^T
    bool f64tc;        // FP64 path with the tensor-core a4 (QMC_PREC_F64_TCA4)
    double kappa_max;  // FP64 recomputation threshold of the float-pair a4
    bool dinv;
    const SysDev *sd;  // the system's sizes
};

size_t al(size_t x) { return (x + 255) & ~size_t(255); }

// c15_override >= 0 replaces the system's c15_mode (qmc_slater_matrices needs all five matrices)
Plan make_plan(const qmc_system *sys, int precision, bool need_dinv, int c15_override = -1)
{
    Plan p;
    const int c15 = c15_override >= 0 ? c15_override : sys->tiles.c15_mode;
    p.msz = (size_t)sys->d.n_up * sys->d.n_up + (size_t)sys->d.n_dn * sys->d.n_dn;
    p.mixed = precision == QMC_PREC_MIXED || precision == QMC_PREC_MIXED_BF16;
    p.f64tc = precision == QMC_PREC_F64_TCA4;
    p.cfree = p.mixed && c15 == QMC_C15_CFREE;
    p.cd_bytes = p.cfree ? (size_t)sys->d.n_elec * 4 * 8 : (p.mixed ? p.msz * (3 * 4 + 8) : p.msz * 4 * 8);
    p.mask_bytes = p.mixed ? (size_t)sys->d.n_elec * sys->mixed.mask_words * 4 : 0;
    p.dinv = need_dinv;
    p.ffgj = (p.mixed && (sys->tiles.a4_mode == QMC_A4_FLOAT_FLOAT || sys->tiles.a4_mode == QMC_A4_TENSOR)) || p.f64tc;
    p.tcgj = (p.mixed && sys->tiles.a4_mode == QMC_A4_TENSOR) ||
             (p.f64tc && gjtc_fits(std::max(sys->d.n_up, sys->d.n_dn)));
    p.kappa_max = p.f64tc ? sys->tiles.f64_kappa_max : sys->tiles.a4_kappa_max;
    p.redo_bytes = p.ffgj ? redo_scratch_bytes(std::max(sys->d.n_up, sys->d.n_dn)) : 0;
    p.c15tc = p.mixed && (c15 == QMC_C15_TENSOR || c15 == QMC_C15_CFREE);
    p.sd = &sys->d;
    p.per_walker = p.msz * 8 + p.cd_bytes + (need_dinv ? p.msz * 8 : 0) + 36 + p.mask_bytes +
                   (p.ffgj ? p.msz * 8 + 2 : 0);
    return p;
}

struct Carve {
    double *X; void *Cd; double *L5; double *D; double *la; double *sg; uint32_t *st; uint32_t *masks;
    float2 *work; uint8_t *redo; void *redo_scratch; void *c15tc; void *gjtc; double *vd; void *vdscr;
};

// Arrays for `nw` walkers laid out array by array inside ws.
bool carve(const Plan &p, int nw, void *ws, size_t ws_bytes, Carve &c)
{
    char *b = static_cast<char *>(ws);
    size_t o = 0;
    auto take = [&](size_t bytes) { char *r = b + o; o = al(o + bytes); return r; };
    c.X = reinterpret_cast<double *>(take(p.msz * 8 * nw));
    c.vd = nullptr;
    c.vdscr = nullptr;
    if (p.cfree) {
        c.Cd = nullptr;
        c.L5 = nullptr;
        c.vd = reinterpret_cast<double *>(take(p.cd_bytes * nw));
        c.vdscr = take(vdrift_bytes(*p.sd, nw));
    } else if (p.mixed) {
        c.Cd = take(p.msz * 3 * 4 * nw);
        c.L5 = reinterpret_cast<double *>(take(p.msz * 8 * nw));
    } else {
        c.Cd = take(p.msz * 4 * 8 * nw);
        c.L5 = nullptr;
    }
    c.D = p.dinv ? reinterpret_cast<double *>(take(p.msz * 8 * nw)) : nullptr;
    c.la = reinterpret_cast<double *>(take(16 * (size_t)nw));
    c.sg = reinterpret_cast<double *>(take(16 * (size_t)nw));
    c.st = reinterpret_cast<uint32_t *>(take(4 * (size_t)nw));
    c.masks = p.mask_bytes ? reinterpret_cast<uint32_t *>(take(p.mask_bytes * nw)) : nullptr;
    // (the tensor-core a4 keeps its work matrices in its own scratch, rows 16-byte aligned)
    c.work = (p.ffgj && !p.tcgj) ? reinterpret_cast<float2 *>(take(p.msz * 8 * nw)) : nullptr;
    c.redo = p.ffgj ? reinterpret_cast<uint8_t *>(take(2 * (size_t)nw)) : nullptr;
    c.redo_scratch = p.ffgj ? take(p.redo_bytes) : nullptr;
    c.c15tc = p.c15tc ? take(c15tc_bytes(*p.sd, nw)) : nullptr;
    c.gjtc = p.tcgj ? take(gjtc_bytes(p.sd->n_up, p.sd->n_dn, nw)) : nullptr;
    return o <= ws_bytes;
}

size_t bytes_for(const Plan &p, int nw)
{
    size_t o = al(p.msz * 8 * nw);
    if (p.cfree) o += al(p.cd_bytes * nw) + al(vdrift_bytes(*p.sd, nw));
    else o += p.mixed ? al(p.msz * 3 * 4 * nw) + al(p.msz * 8 * nw) : al(p.msz * 4 * 8 * nw);
    o += p.dinv ? al(p.msz * 8 * nw) : 0;
    o += al(16 * (size_t)nw) * 2 + al(4 * (size_t)nw);
    o += p.mask_bytes ? al(p.mask_bytes * nw) : 0;
    o += (p.ffgj && !p.tcgj) ? al(p.msz * 8 * nw) : 0;
    o += p.ffgj ? al(2 * (size_t)nw) + al(p.redo_bytes) : 0;
    o += p.c15tc ? al(c15tc_bytes(*p.sd, nw)) : 0;
    o += p.tcgj ? al(gjtc_bytes(p.sd->n_up, p.sd->n_dn, nw)) : 0;
    return o;
}

int chunk_walkers(const Plan &p, int W, size_t ws_bytes)
{
    int lo = 0, hi = std::min(W, 65535);
    while (lo < hi) {
        const int mid = lo + (hi - lo + 1) / 2;
        if (bytes_for(p, mid) <= ws_bytes) lo = mid; else hi = mid - 1;
    }
    return lo;
}

CView cview(const Plan &p, const Carve &c)
{
    CView v;
    v.g = c.Cd;
    v.vd = c.vd;
    if (p.cfree) {
        v.g_f32 = 1; v.g_wstride = 0; v.g_ncomp = 3;
        v.l = nullptr; v.l_wstride = 0; v.l_ncomp = 1; v.l_comp = 0;
    } else if (p.mixed) {
        v.g_f32 = 1; v.g_wstride = 3 * p.msz; v.g_ncomp = 3;
        v.l = c.L5; v.l_wstride = p.msz; v.l_ncomp = 1; v.l_comp = 0;
    } else {
        v.g_f32 = 0; v.g_wstride = 4 * p.msz; v.g_ncomp = 4;
        v.l = static_cast<const double *>(c.Cd); v.l_wstride = 4 * p.msz; v.l_ncomp = 4; v.l_comp = 3;
    }
    return v;
}

// Steps a1-a3 for one chunk of walkers: C1 -> c.X (FP64), C2..C5 -> c.Cd
// (FP64 in the FP64 path, FP32 in the mixed path).
// `mark(q)` (if set) records event q after product kernel q-4 (mask, C1/C5, tensor cores).
// The bounded-wait settings of one walker chunk starting at walker w0.
WaitCfg wait_cfg(const qmc_system *sys, int w0, int nw)
{
    WaitCfg wc;
    wc.limit_ns = (unsigned long long)(sys->tiles.wait_s * 1e9);
    const int x = sys->tiles.expire_walker;
    wc.expire_w = (x >= w0 && x < w0 + nw) ? x - w0 : -1;
    wc.expire_kernels = sys->tiles.expire_kernels;
    return wc;
}

template <typename Mark>
cudaError_t run_products(const qmc_system *sys, int precision, int nw, const double *Rc, const Carve &c,
                         cudaStream_t st, Mark mark, const WaitCfg &wc, const Plan &p)
{
    const SysDev &s = sys->d;
    if (!p.mixed) return launch_contract_f64(s, nw, Rc, c.X, static_cast<double *>(c.Cd), st);
    const MixedTables &mt = sys->mixed;
    cudaError_t e = launch_shell_mask(s, mt, nw, Rc, mt.mask_words, c.masks, st);
    if (e != cudaSuccess) return e;
    if ((e = mark(4)) != cudaSuccess) return e;
    TcTables tt;
    tt.f16 = precision == QMC_PREC_MIXED ? 1 : 0;
    for (int spin = 0; spin < 2; ++spin) {
        tt.hi[spin] = tt.f16 ? mt.hhi[spin] : mt.bhi[spin];
        tt.lo[spin] = tt.f16 ? mt.hlo[spin] : mt.blo[spin];
        tt.ns_pad[spin] = mt.ns_pad[spin];
        for (int l = 0; l < 3; ++l)
            tt.out_scale[spin][l] = tt.f16 ? (float)ldexp(1.0, -(mt.a_exp[spin] + mt.b_exp)) : 1.0f;
    }
    for (int l = 0; l < 3; ++l) tt.in_scale[l] = tt.f16 ? (float)ldexp(1.0, mt.b_exp) : 1.0f;
    tt.pgf = mt.pgf; tt.pcf = mt.pcf; tt.scf = mt.scf; tt.Qhi = mt.Qhi; tt.Qlo = mt.Qlo;
    if (p.cfree) {
        // the C-free variant: C1 alone here; drift and Laplacian after a4 (launch_vdrift)
        e = launch_c15_tc(s, mt.ffb, mt, tt, nw, Rc, c.masks, mt.mask_words, c.X, nullptr, nullptr, c.st, c.c15tc,
                          st, wc, true);
        if (e != cudaSuccess) return e;
        return mark(5);
    }
    if (p.c15tc) {
        // C1, C5 and C2..C4 from one producer pass per (electron, walker tile)
        e = launch_c15_tc(s, mt.ffb, mt, tt, nw, Rc, c.masks, mt.mask_words, c.X, c.L5,
                          static_cast<float *>(c.Cd), c.st, c.c15tc, st, wc);
        if (e != cudaSuccess) return e;
        return mark(5);
    }
    e = launch_c15_ff(s, mt.ffb, nw, Rc, c.masks, mt.mask_words, mt.ff, mt.ns32, mt.colmax, c.X, c.L5, st,
                      sys->tiles.c15_walkers);
    if (e != cudaSuccess) return e;
    if ((e = mark(5)) != cudaSuccess) return e;
    return launch_tc_contract(s, nw, Rc, c.masks, mt.mask_words, tt, static_cast<float *>(c.Cd), c.st, st, wc);
}


}  // namespace

extern "C" int qmc_workspace_size(const qmc_system *sys, int n_walk, int precision, size_t *bytes)
{
    if (!sys || !bytes || n_walk < 0) return invalid("qmc_workspace_size: bad argument");
    if (precision < QMC_PREC_F64 || precision > QMC_PREC_F64_TCA4) return invalid("qmc_workspace_size: precision");
    const Plan p = make_plan(sys, precision, true);
    *bytes = bytes_for(p, std::min(n_walk, 65535));
    return QMC_OK;
}

namespace {

// Events bracketing the three stages of one evaluation (contraction a1-a3,
// inverse a4, energies a5-a6); created on first use per thread.
struct StageEvents {
    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int device = -1;
    ~StageEvents()
    {
        for (auto &e : ev) if (e) cudaEventDestroy(e);
    }
    cudaError_t ensure(int dev)
    {
        if (device == dev && ev[0]) return cudaSuccess;
        for (auto &e : ev) {
            if (e) cudaEventDestroy(e);
            e = nullptr;
            cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) return r;
        }
        device = dev;
        return cudaSuccess;
    }
};
thread_local StageEvents t_events;

int eval_impl(const qmc_system *sys, int n_walk, const double *R, int precision, const qmc_eval_out *out, void *ws,
              size_t ws_bytes, cudaStream_t st, float *stage_ms)
{
    if (!sys || !out) return invalid("qmc_walkers_eval: null argument");
    if (n_walk < 0) return invalid("qmc_walkers_eval: n_walk < 0");
    if (stage_ms) for (int q = 0; q < 8; ++q) stage_ms[q] = 0.0f;
    if (n_walk == 0) return QMC_OK;
    if (!R || !out->logpsi || !out->sign || !out->drift || !out->e_loc || !out->status)
        return invalid("qmc_walkers_eval: null required pointer");
    if (precision < QMC_PREC_F64 || precision > QMC_PREC_F64_TCA4) return invalid("qmc_walkers_eval: precision");
    const Plan p = make_plan(sys, precision, out->dinv == nullptr);
    const int chunk = chunk_walkers(p, n_walk, ws_bytes);
    if (chunk < 1) {
        set_error("qmc_walkers_eval: workspace smaller than one walker");
        return QMC_ERR_CAPACITY;
    }
    const SysDev &s = sys->d;
    cudaError_t e = cudaSetDevice(sys->device);
    if (e != cudaSuccess) return cuda_fail(e, "qmc_walkers_eval: cudaSetDevice");
    if (stage_ms) {
        e = t_events.ensure(sys->device);
        if (e != cudaSuccess) return cuda_fail(e, "qmc_walkers_eval: event create");
    }
    auto mark = [&](int q) -> cudaError_t { return stage_ms ? cudaEventRecord(t_events.ev[q], st) : cudaSuccess; };
    for (int w0 = 0; w0 < n_walk; w0 += chunk) {
        const int nw = std::min(chunk, n_walk - w0);
        Carve c;
        carve(p, nw, ws, ws_bytes, c);
        const double *Rc = R + (size_t)w0 * s.n_elec * 3;
        double *Dinv = out->dinv ? out->dinv + (size_t)w0 * p.msz : c.D;
        if ((e = mark(0)) != cudaSuccess) return cuda_fail(e, "qmc_walkers_eval: event");
        e = cudaMemsetAsync(c.st, 0, 4 * (size_t)nw, st);
        if (e != cudaSuccess) return cuda_fail(e, "qmc_walkers_eval: memset");
        const WaitCfg wc = wait_cfg(sys, w0, nw);
        e = run_products(sys, precision, nw, Rc, c, st, mark, wc, p);
        if (e != cudaSuccess) return cuda_fail(e, "qmc_walkers_eval: products launch");
        if ((e = mark(1)) != cudaSuccess) return cuda_fail(e, "qmc_walkers_eval: event");
        GjJob jobs[2] = {GjJob(), GjJob()};
        int nj = 0;
        for (int spin = 0; spin < 2; ++spin) {
            const int ns = spin ? s.n_dn : s.n_up;
            if (ns == 0) continue;
            const size_t off = spin ? (size_t)s.n_up * s.n_up : 0;
            GjJob &j = jobs[nj++];
            j.X = c.X + off; j.x_stride = (long long)p.msz;
            j.Dinv = Dinv + off; j.d_stride = (long long)p.msz;
            j.logabs = c.la + spin; j.la_stride = 2;
            j.sign = c.sg + spin;
            j.flag = c.st; j.flag_bit = spin ? QMC_STATUS_SINGULAR_DN : QMC_STATUS_SINGULAR_UP;
            j.n = ns; j.count = nw;
            if (p.ffgj) { j.work = c.work ? c.work + off : nullptr; j.redo = c.redo + spin; j.redo_stride = 2; }
        }
        if (p.ffgj) {
            // float-pair elimination for every matrix, FP64 for those it flags
            e = cudaMemsetAsync(c.redo, 0, 2 * (size_t)nw, st);
            if (e != cudaSuccess) return cuda_fail(e, "qmc_walkers_eval: memset");
            GjJob ffj[2] = {jobs[0], jobs[1]};
            for (int q = 0; q < nj; ++q) ffj[q].flag = nullptr;
            if (p.tcgj) e = launch_gj_tc(ffj, nj, c.gjtc, st, p.kappa_max, wc);
            else e = launch_gj_ff(ffj, nj, st, sys->tiles.gj_panel, p.kappa_max);
            if (e != cudaSuccess) return cuda_fail(e, "qmc_walkers_eval: float-float Gauss-Jordan launch");
            if (!p.f64tc) {
                // near-node matrices: C1 again in FP64 (the mixed C1 carries its ~2^-40 error), then
                // the FP64 elimination, multi-CTA for the first kRedoMax of them
                int e_off[2], q = 0;
                for (int spin = 0; spin < 2; ++spin)
                    if (spin ? s.n_dn : s.n_up) e_off[q++] = spin ? s.n_up : 0;
                e = launch_gj_redo(jobs, nj, c.redo_scratch, st, sys->tiles.gj_panel, &s, Rc, e_off);
                if (e != cudaSuccess) return cuda_fail(e, "qmc_walkers_eval: FP64 recomputation launch");
            }
            // (QMC_PREC_F64_TCA4: C1 is FP64 already; every flagged matrix goes to the batched
            // FP64 elimination below, one CTA per matrix)
            for (int q = 0; q < nj; ++q) jobs[q].only_redo = 1;
        }
        e = launch_gj(jobs, nj, st, sys->tiles.gj_panel);
        if (e != cudaSuccess) return cuda_fail(e, "qmc_walkers_eval: Gauss-Jordan launch");
        if ((e = mark(2)) != cudaSuccess) return cuda_fail(e, "qmc_walkers_eval: event");
        if (p.cfree) {
            e = launch_vdrift(s, sys->mixed.ffb, sys->mixed, nw, Rc, c.masks, sys->mixed.mask_words, Dinv, c.vd, c.st,
                              c.vdscr, st, wc);
            if (e != cudaSuccess) return cuda_fail(e, "qmc_walkers_eval: C-free drift launch");
        }
        e = launch_drift_energy(s, nw, Rc, Dinv, cview(p, c), c.la, c.sg, c.st, *out, w0, st, sys->mixed.ffb.Q);
        if (e != cudaSuccess) return cuda_fail(e, "qmc_walkers_eval: energy launch");
        if (stage_ms) {
            if ((e = mark(3)) != cudaSuccess) return cuda_fail(e, "qmc_walkers_eval: event");
            if ((e = cudaEventSynchronize(t_events.ev[3])) != cudaSuccess)
                return cuda_fail(e, "qmc_walkers_eval: event sync");
            for (int q = 0; q < 3; ++q) {
                float ms = 0.0f;
                if ((e = cudaEventElapsedTime(&ms, t_events.ev[q], t_events.ev[q + 1])) != cudaSuccess)
                    return cuda_fail(e, "qmc_walkers_eval: elapsed");
                stage_ms[q] += ms;
                stage_ms[3] += ms;
            }
            if (p.mixed) {   // split of stage 0 into its three kernels
                float m4 = 0.0f, m5 = 0.0f, m6 = 0.0f;
                if ((e = cudaEventElapsedTime(&m4, t_events.ev[0], t_events.ev[4])) != cudaSuccess ||
                    (e = cudaEventElapsedTime(&m5, t_events.ev[4], t_events.ev[5])) != cudaSuccess ||
                    (e = cudaEventElapsedTime(&m6, t_events.ev[5], t_events.ev[1])) != cudaSuccess)
                    return cuda_fail(e, "qmc_walkers_eval: elapsed");
                stage_ms[4] += m4; stage_ms[5] += m5; stage_ms[6] += m6;
            } else {
                stage_ms[5] += stage_ms[0];
            }
        }
    }
    return QMC_OK;
}

}  // namespace

extern "C" int qmc_walkers_eval(const qmc_system *sys, int n_walk, const double *R, int precision,
                                const qmc_eval_out *out, void *ws, size_t ws_bytes, qmc_stream_t stream)
{
    return eval_impl(sys, n_walk, R, precision, out, ws, ws_bytes, reinterpret_cast<cudaStream_t>(stream), nullptr);
}

extern "C" int qmc_walkers_eval_timed(const qmc_system *sys, int n_walk, const double *R, int precision,
                                      const qmc_eval_out *out, void *ws, size_t ws_bytes, qmc_stream_t stream,
                                      float *stage_ms)
{
    if (!stage_ms) return invalid("qmc_walkers_eval_timed: stage_ms is null");
    return eval_impl(sys, n_walk, R, precision, out, ws, ws_bytes, reinterpret_cast<cudaStream_t>(stream), stage_ms);
}

extern "C" int qmc_slater_matrices(const qmc_system *sys, int n_walk, const double *R, int precision, double *C,
                                   void *ws, size_t ws_bytes, qmc_stream_t stream)
{
    if (!sys || (n_walk > 0 && (!R || !C))) return invalid("qmc_slater_matrices: null argument");
    if (n_walk < 0) return invalid("qmc_slater_matrices: n_walk < 0");
    if (precision < QMC_PREC_F64 || precision > QMC_PREC_F64_TCA4) return invalid("qmc_slater_matrices: precision");
    if (n_walk == 0) return QMC_OK;
    // all five matrices: the C-free variant's system computes them as the tensor-core mode does
    const Plan p = make_plan(sys, precision, false,
                             sys->tiles.c15_mode == QMC_C15_CFREE ? QMC_C15_TENSOR : sys->tiles.c15_mode);
    const int chunk = chunk_walkers(p, n_walk, ws_bytes);
    if (chunk < 1) {
        set_error("qmc_slater_matrices: workspace smaller than one walker");
        return QMC_ERR_CAPACITY;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const SysDev &s = sys->d;
    cudaError_t e = cudaSetDevice(sys->device);
    if (e != cudaSuccess) return cuda_fail(e, "qmc_slater_matrices: cudaSetDevice");
    const size_t nu2 = (size_t)s.n_up * s.n_up, nd2 = (size_t)s.n_dn * s.n_dn;
    const size_t opitch = 5 * p.msz * sizeof(double);
    for (int w0 = 0; w0 < n_walk; w0 += chunk) {
        const int nw = std::min(chunk, n_walk - w0);
        Carve c;
        carve(p, nw, ws, ws_bytes, c);
        const double *Rc = R + (size_t)w0 * s.n_elec * 3;
        e = cudaMemsetAsync(c.st, 0, 4 * (size_t)nw, st);
        if (e != cudaSuccess) return cuda_fail(e, "qmc_slater_matrices: memset");
        e = run_products(sys, precision, nw, Rc, c, st, [](int) { return cudaSuccess; }, wait_cfg(sys, w0, nw), p);
        if (e != cudaSuccess) return cuda_fail(e, "qmc_slater_matrices: products launch");
        char *o = reinterpret_cast<char *>(C + (size_t)w0 * 5 * p.msz);
        // per walker: [C1 up][C2..C5 up][C1 dn][C2..C5 dn]
        const size_t xs[2] = {0, nu2}, ws2[2] = {nu2, nd2}, os[2] = {0, 5 * nu2};
        for (int spin = 0; spin < 2; ++spin) {
            if (ws2[spin] == 0) continue;
            e = cudaMemcpy2DAsync(o + os[spin] * 8, opitch, c.X + xs[spin], p.msz * 8, ws2[spin] * 8, nw,
                                  cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return cuda_fail(e, "qmc_slater_matrices: copy");
            double *dst = reinterpret_cast<double *>(o) + os[spin] + ws2[spin];
            if (!p.mixed) {
                e = cudaMemcpy2DAsync(dst, opitch, static_cast<double *>(c.Cd) + 4 * xs[spin], 4 * p.msz * 8,
                                      4 * ws2[spin] * 8, nw, cudaMemcpyDeviceToDevice, st);
            } else {
                e = launch_widen(static_cast<float *>(c.Cd) + 3 * xs[spin], 3 * p.msz, dst, 5 * p.msz, 3 * ws2[spin],
                                 nw, st);
                if (e == cudaSuccess)
                    e = cudaMemcpy2DAsync(dst + 3 * ws2[spin], opitch, c.L5 + xs[spin], p.msz * 8, ws2[spin] * 8,
                                          nw, cudaMemcpyDeviceToDevice, st);
            }
            if (e != cudaSuccess) return cuda_fail(e, "qmc_slater_matrices: copy");
        }
    }
    return QMC_OK;
}

extern "C" int qmc_det_inverse(int batch, int n, double *X, double *Dinv, double *logabs, double *sign,
                               uint32_t *singular, qmc_stream_t stream)
{
    if (batch < 0 || n < 1 || n > kMaxN) return invalid("qmc_det_inverse: need batch >= 0 and 1 <= n <= 1024");
    if (batch == 0) return QMC_OK;
    if (!X || !Dinv) return invalid("qmc_det_inverse: null matrix pointer");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    GjJob j = GjJob();
    j.X = X; j.x_stride = (long long)n * n;
    j.Dinv = Dinv; j.d_stride = (long long)n * n;
    j.logabs = logabs; j.la_stride = 1;
    j.sign = sign;
    j.flag = singular; j.flag_bit = 1u;
    j.n = n; j.count = batch;
    if (singular) {
        cudaError_t e = cudaMemsetAsync(singular, 0, sizeof(uint32_t) * batch, st);
        if (e != cudaSuccess) return cuda_fail(e, "qmc_det_inverse: memset");
    }
    cudaError_t e = launch_gj(&j, 1, st, n > 640 ? 8 : 16);
    if (e != cudaSuccess) return cuda_fail(e, "qmc_det_inverse: launch");
    return QMC_OK;
}

extern "C" int qmc_screen_ao(const qmc_system *sys, int n_walk, const double *R, int cap, int32_t *cnt,
                             int32_t *idx, double *B, qmc_stream_t stream)
{
    if (!sys || n_walk < 0 || cap < 0) return invalid("qmc_screen_ao: bad argument");
    if (n_walk == 0) return QMC_OK;
    if (!R || !cnt || (cap > 0 && !idx)) return invalid("qmc_screen_ao: null pointer");
    if (n_walk > 65535) return invalid("qmc_screen_ao: at most 65535 walkers per call");
    cudaError_t e = launch_screen_ao(sys->d, n_walk, R, cap, cnt, idx, B, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "qmc_screen_ao: launch");
    return QMC_OK;
}

extern "C" int qmc_shell_masks(const qmc_system *sys, int n_walk, const double *R, uint32_t *masks,
                               int *mask_words, qmc_stream_t stream)
{
    if (!sys || n_walk < 0 || !mask_words) return invalid("qmc_shell_masks: bad argument");
    *mask_words = sys->mixed.mask_words;
    if (!masks || n_walk == 0) return QMC_OK;
    if (!R) return invalid("qmc_shell_masks: null pointer");
    if (n_walk > 65535) return invalid("qmc_shell_masks: at most 65535 walkers per call");
    cudaError_t e = launch_shell_mask(sys->d, sys->mixed, n_walk, R, sys->mixed.mask_words, masks,
                                      reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "qmc_shell_masks: launch");
    return QMC_OK;
}

extern "C" int qmc_logpsi_backward(const qmc_system *sys, int n_walk, const double *R, const double *dinv,
                                   const double *g, double *dA_up, double *dA_dn, qmc_stream_t stream)
{
    if (!sys || n_walk < 0) return invalid("qmc_logpsi_backward: bad argument");
    if (!dA_up || !dA_dn || (n_walk > 0 && (!R || !dinv || !g))) return invalid("qmc_logpsi_backward: null pointer");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = launch_backward_f64(sys->d, n_walk, R, dinv, g, dA_up, dA_dn, st, sys->max_shell_per_atom);
    if (e != cudaSuccess) return cuda_fail(e, "qmc_logpsi_backward: launch");
    return QMC_OK;
}

extern "C" int qmc_backward_workspace_size(const qmc_system *sys, int n_walk, int precision, size_t *bytes)
{
    if (!sys || n_walk < 0 || !bytes) return invalid("qmc_backward_workspace_size: bad argument");
    if (precision == QMC_PREC_F64 || precision == QMC_PREC_F64_TCA4) {
        *bytes = 0;
        return QMC_OK;
    }
    if (precision != QMC_PREC_MIXED) return invalid("qmc_backward_workspace_size: precision");
    *bytes = bwtc_bytes(sys->d, sys->mixed.mask_words, n_walk, sys->tiles.bw_walkers);
    return QMC_OK;
}

extern "C" int qmc_logpsi_backward_ex(const qmc_system *sys, int n_walk, const double *R, const double *dinv,
                                      const double *g, int precision, double *dA_up, double *dA_dn, void *ws,
                                      size_t ws_bytes, qmc_stream_t stream)
{
    if (precision == QMC_PREC_F64 || precision == QMC_PREC_F64_TCA4)
        return qmc_logpsi_backward(sys, n_walk, R, dinv, g, dA_up, dA_dn, stream);
    if (!sys || n_walk < 0) return invalid("qmc_logpsi_backward_ex: bad argument");
    if (precision != QMC_PREC_MIXED) return invalid("qmc_logpsi_backward_ex: precision");
    if (!dA_up || !dA_dn || (n_walk > 0 && (!R || !dinv || !g || !ws)))
        return invalid("qmc_logpsi_backward_ex: null pointer");
    if (sys->bw.nb == 0 || sys->bw.nblk == 0) return invalid("qmc_logpsi_backward_ex: no AO blocks");
    cudaError_t e = cudaSetDevice(sys->device);
    if (e != cudaSuccess) return cuda_fail(e, "qmc_logpsi_backward_ex: cudaSetDevice");
    e = launch_backward_tc(sys->d, sys->mixed, sys->bw, sys->tiles.bw_walkers, n_walk, R, dinv, g, dA_up, dA_dn,
                           ws, ws_bytes, reinterpret_cast<cudaStream_t>(stream), wait_cfg(sys, 0, n_walk));
    if (e == cudaErrorMemoryAllocation) {
        set_error("qmc_logpsi_backward_ex: workspace smaller than one walker");
        return QMC_ERR_CAPACITY;
    }
    if (e != cudaSuccess) return cuda_fail(e, "qmc_logpsi_backward_ex: launch");
    return QMC_OK;
}

// ---------------------------------------------------------------------------
// Walker evaluation without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs under a memory manager
// owning all device memory (a framework's caching allocator that must not be
// bypassed), code in a latency-critical loop where cudaMalloc's implicit
// device synchronisation is not acceptable, or a plug-in inside a host
// application that forbids driver allocations.  For them the scratch of
// qmc_walkers_eval lives in the fixed array below, which every device that
// loads this library holds until the process exits.
namespace {

constexpr size_t kStaticScratchBytes = (size_t)QMC_STATIC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;

// Device address of the array per device, with the id of the CUDA context it
// was looked up in: if the context is destroyed and recreated (a
// cudaDeviceReset elsewhere in the process), the module is loaded again and the
// array may move, so a changed id means looking it up again.
struct StaticSlot {
    unsigned long long ctx_id = 0;
    void *ptr = nullptr;
};
StaticSlot g_static_slot[kMaxDevices];
std::mutex g_static_mutex;

// Id of the calling thread's current CUDA context, through driver entry points
// the runtime hands out (so the library needs no link against libcuda).
cudaError_t current_ctx_id(unsigned long long *id)
{
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    if (!get_current || !get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 4000, cudaEnableDefault, &q1);
        if (e == cudaSuccess) e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e != cudaSuccess) return e;
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return cudaErrorSymbolNotFound;
        get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f1);
        get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(f2);
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
    return cudaSuccess;
}

}  // namespace

extern "C" int qmc_walkers_eval_static(const qmc_system *sys, int n_walk, const double *R, int precision,
                                       const qmc_eval_out *out, qmc_stream_t stream)
{
    if (!sys || !out) return invalid("qmc_walkers_eval_static: null argument");
    if (n_walk < 0) return invalid("qmc_walkers_eval_static: n_walk < 0");
    if (n_walk == 0) return QMC_OK;
    const int dev = sys->device;
    if (dev < 0 || dev >= kMaxDevices) return invalid("qmc_walkers_eval_static: device index out of range");
    if (precision < QMC_PREC_F64 || precision > QMC_PREC_F64_TCA4)
        return invalid("qmc_walkers_eval_static: precision");
    const Plan p = make_plan(sys, precision, out->dinv == nullptr);
    if (bytes_for(p, 1) > kStaticScratchBytes) {
        set_error("qmc_walkers_eval_static: one walker of this system needs " + std::to_string(bytes_for(p, 1)) +
                  " bytes of scratch, more than the library's fixed " + std::to_string(kStaticScratchBytes) +
                  "-byte array; use qmc_walkers_eval with a caller workspace");
        return QMC_ERR_CAPACITY;
    }
    cudaError_t e = cudaSetDevice(dev);
    if (e != cudaSuccess) return cuda_fail(e, "qmc_walkers_eval_static: cudaSetDevice");
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_static_mutex);
        // the context now current for this device (cudaSetDevice made its primary context current)
        unsigned long long ctx_id = 0;
        e = current_ctx_id(&ctx_id);
        if (e != cudaSuccess) return cuda_fail(e, "qmc_walkers_eval_static: current context id");
        StaticSlot &slot = g_static_slot[dev];
        if (!slot.ptr || slot.ctx_id != ctx_id) {
            // first call on this device (or in a new context): the host-side
            // symbol is only a stand-in, the kernels need the array's device address
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_static_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "qmc_walkers_eval_static: cudaGetSymbolAddress");
            slot.ptr = ptr;
            slot.ctx_id = ctx_id;
        }
        scratch = slot.ptr;
    }
    return eval_impl(sys, n_walk, R, precision, out, scratch, kStaticScratchBytes,
                     reinterpret_cast<cudaStream_t>(stream), nullptr);
}

// ---------------------------------------------------------------------------
// Multi-determinant expansion (Sec. II.C, Eq. psit): the determinants one after the
// other with the same evaluation, then their combination.
namespace {

struct MdCarve {
    double *lp, *sg, *el, *ep, *dr;
    uint32_t *st;
    char *eval_ws;
    size_t eval_bytes;
};

size_t md_own_bytes(int K, int W, int N)
{
    return 3 * al((size_t)K * W * 8) + al((size_t)K * W * 32) + al((size_t)K * W * N * 24) + al((size_t)K * W * 4);
}

int md_check(const qmc_system *const *dets, int n_det, int precision, const char *who)
{
    if (!dets || n_det < 1 || n_det > kMaxDets) return invalid(std::string(who) + ": need 1..64 determinants");
    if (precision < QMC_PREC_F64 || precision > QMC_PREC_F64_TCA4) return invalid(std::string(who) + ": precision");
    for (int k = 0; k < n_det; ++k) {
        const qmc_system *a = dets[k], *b = dets[0];
        if (!a) return invalid(std::string(who) + ": null determinant");
        if (a->device != b->device || a->d.n_up != b->d.n_up || a->d.n_dn != b->d.n_dn || a->d.n_atom != b->d.n_atom ||
            a->d.n_ao != b->d.n_ao)
            return invalid(std::string(who) + ": determinants must share the device, electrons, atoms and basis");
        if (a->d.jas != b->d.jas || (a->d.jas && (a->d.ja_par != b->d.ja_par || a->d.ja_anti != b->d.ja_anti ||
                                                  a->d.jb_ee != b->d.jb_ee)))
            return invalid(std::string(who) + ": determinants must carry the same Jastrow factor");
    }
    return QMC_OK;
}

}  // namespace

extern "C" int qmc_multidet_workspace_size(const qmc_system *const *dets, int n_det, int n_walk, int precision,
                                           size_t *bytes)
{
    int rc = md_check(dets, n_det, precision, "qmc_multidet_workspace_size");
    if (rc) return rc;
    if (!bytes || n_walk < 0) return invalid("qmc_multidet_workspace_size: bad argument");
    size_t ev = 0;
    for (int k = 0; k < n_det; ++k) ev = std::max(ev, bytes_for(make_plan(dets[k], precision, true), std::min(n_walk, 65535)));
    *bytes = md_own_bytes(n_det, n_walk, dets[0]->d.n_elec) + ev;
    return QMC_OK;
}

extern "C" int qmc_multidet_eval(const qmc_system *const *dets, const double *coef, int n_det, int n_walk,
                                 const double *R, int precision, const qmc_eval_out *out, void *ws, size_t ws_bytes,
                                 qmc_stream_t stream)
{
    int rc = md_check(dets, n_det, precision, "qmc_multidet_eval");
    if (rc) return rc;
    if (!coef || !out || n_walk < 0) return invalid("qmc_multidet_eval: bad argument");
    if (n_walk == 0) return QMC_OK;
    if (!R || !out->logpsi || !out->sign || !out->drift || !out->e_loc || !out->status || !ws)
        return invalid("qmc_multidet_eval: null required pointer");
    if (out->dinv) return invalid("qmc_multidet_eval: no single D^-1 exists for an expansion (pass dinv = NULL)");
    const int N = dets[0]->d.n_elec, W = n_walk, K = n_det;
    char *b = static_cast<char *>(ws);
    size_t o = 0;
    auto take = [&](size_t bytes) { char *r = b + o; o = al(o + bytes); return r; };
    MdCarve c;
    c.lp = reinterpret_cast<double *>(take((size_t)K * W * 8));
    c.sg = reinterpret_cast<double *>(take((size_t)K * W * 8));
    c.el = reinterpret_cast<double *>(take((size_t)K * W * 8));
    c.ep = reinterpret_cast<double *>(take((size_t)K * W * 32));
    c.dr = reinterpret_cast<double *>(take((size_t)K * W * N * 24));
    c.st = reinterpret_cast<uint32_t *>(take((size_t)K * W * 4));
    if (o > ws_bytes) {
        set_error("qmc_multidet_eval: workspace below qmc_multidet_workspace_size");
        return QMC_ERR_CAPACITY;
    }
    c.eval_ws = b + o;
    c.eval_bytes = ws_bytes - o;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    for (int k = 0; k < K; ++k) {
        qmc_eval_out eo;
        memset(&eo, 0, sizeof eo);
        eo.logpsi = c.lp + (size_t)k * W;
        eo.sign = c.sg + (size_t)k * W;
        eo.e_loc = c.el + (size_t)k * W;
        eo.e_parts = c.ep + (size_t)k * W * 4;
        eo.drift = c.dr + (size_t)k * W * N * 3;
        eo.status = c.st + (size_t)k * W;
        rc = eval_impl(dets[k], W, R, precision, &eo, c.eval_ws, c.eval_bytes, st, nullptr);
        if (rc) return rc;
    }
    cudaError_t e = launch_multidet_combine(W, N, K, coef, c.lp, c.sg, c.dr, c.el, c.ep, c.st, *out, st);
    if (e != cudaSuccess) return cuda_fail(e, "qmc_multidet_eval: combine launch");
    return QMC_OK;
}

// ---------------------------------------------------------------------------
// The Monte Carlo step (Sec. II.A, II.B).
namespace {

constexpr int kMaxSrmcWalkers = 1 << 24;

struct DmcCarve {
    double *R, *drift, *e, *lp, *sg, *w;
    uint32_t *st, *acc;
    int *idx;
    unsigned long long *C;
    char *eval_ws;
    size_t eval_bytes;
};

size_t dmc_own_bytes(int W, int n_elec)
{
    const size_t nc = (size_t)W * n_elec * 3;
    return 2 * al(nc * 8) + 4 * al((size_t)W * 8) + 2 * al((size_t)W * 4) + al((size_t)W * 4) + al((size_t)W * 8);
}

bool dmc_carve(int W, int n_elec, void *ws, size_t ws_bytes, DmcCarve &c)
{
    char *b = static_cast<char *>(ws);
    size_t o = 0;
    auto take = [&](size_t bytes) { char *r = b + o; o = al(o + bytes); return r; };
    const size_t nc = (size_t)W * n_elec * 3;
    c.R = reinterpret_cast<double *>(take(nc * 8));
    c.drift = reinterpret_cast<double *>(take(nc * 8));
    c.e = reinterpret_cast<double *>(take((size_t)W * 8));
    c.lp = reinterpret_cast<double *>(take((size_t)W * 8));
    c.sg = reinterpret_cast<double *>(take((size_t)W * 8));
    c.w = reinterpret_cast<double *>(take((size_t)W * 8));
    c.st = reinterpret_cast<uint32_t *>(take((size_t)W * 4));
    c.acc = reinterpret_cast<uint32_t *>(take((size_t)W * 4));
    c.idx = reinterpret_cast<int *>(take((size_t)W * 4));
    c.C = reinterpret_cast<unsigned long long *>(take((size_t)W * 8));
    if (o > ws_bytes) return false;
    c.eval_ws = b + o;
    c.eval_bytes = ws_bytes - o;
    return true;
}

bool state_ok(const qmc_walker_state *s)
{
    return s && s->R && s->drift && s->e_loc && s->logpsi && s->sign && s->status;
}

}  // namespace

extern "C" int qmc_dmc_move(int n_walk, int n_elec, const double *R, const double *drift, double tau, uint64_t seed,
                            uint64_t step, const uint64_t *step_ptr, double *R_new, qmc_stream_t stream)
{
    if (n_walk < 0 || n_elec < 0) return invalid("qmc_dmc_move: negative size");
    if (!(tau > 0.0) || !isfinite(tau)) return invalid("qmc_dmc_move: tau must be positive and finite");
    if (n_walk == 0 || n_elec == 0) return QMC_OK;
    if (!R || !drift || !R_new) return invalid("qmc_dmc_move: null pointer");
    if (R_new == R) return invalid("qmc_dmc_move: R_new may not alias R");
    cudaError_t e = launch_dmc_move(n_walk, n_elec, R, drift, tau, seed, step, step_ptr, R_new,
                                    reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "qmc_dmc_move: launch");
    return QMC_OK;
}

extern "C" int qmc_dmc_weight(int n_walk, const double *e_old, const double *sign_old, const uint32_t *status_old,
                              const double *e_new, const double *sign_new, const uint32_t *status_new, double tau,
                              double e_trial, const double *e_trial_ptr, double *weight, uint32_t *accept,
                              qmc_stream_t stream)
{
    if (n_walk < 0) return invalid("qmc_dmc_weight: n_walk < 0");
    if (!(tau > 0.0) || !isfinite(tau)) return invalid("qmc_dmc_weight: tau must be positive and finite");
    if (n_walk == 0) return QMC_OK;
    if (!e_old || !sign_old || !status_old || !e_new || !sign_new || !status_new || !weight || !accept)
        return invalid("qmc_dmc_weight: null pointer");
    cudaError_t e = launch_dmc_weight(n_walk, e_old, sign_old, status_old, e_new, sign_new, status_new, tau, e_trial,
                                      e_trial_ptr, weight, accept, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "qmc_dmc_weight: launch");
    return QMC_OK;
}

extern "C" int qmc_srmc_reconfigure(int n_walk, const double *weight, uint64_t seed, uint64_t step,
                                    const uint64_t *step_ptr, int32_t *idx, double *stats, void *ws, size_t ws_bytes,
                                    qmc_stream_t stream)
{
    if (n_walk < 0 || n_walk > kMaxSrmcWalkers) return invalid("qmc_srmc_reconfigure: need 0 <= n_walk <= 2^24");
    if (n_walk == 0) return QMC_OK;
    if (!weight || !idx || !ws) return invalid("qmc_srmc_reconfigure: null pointer");
    if (ws_bytes < (size_t)n_walk * 8) {
        set_error("qmc_srmc_reconfigure: scratch below 8 bytes per walker");
        return QMC_ERR_CAPACITY;
    }
    if (reinterpret_cast<uintptr_t>(ws) & 7) return invalid("qmc_srmc_reconfigure: scratch not 8-byte aligned");
    cudaError_t e = launch_srmc(n_walk, weight, seed, step, step_ptr, static_cast<unsigned long long *>(ws), idx,
                                stats, nullptr, nullptr, nullptr, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "qmc_srmc_reconfigure: launch");
    return QMC_OK;
}

extern "C" int qmc_dmc_workspace_size(const qmc_system *sys, int n_walk, int precision, size_t *bytes)
{
    if (!sys || !bytes || n_walk < 0) return invalid("qmc_dmc_workspace_size: bad argument");
    if (precision < QMC_PREC_F64 || precision > QMC_PREC_F64_TCA4) return invalid("qmc_dmc_workspace_size: precision");
    const Plan p = make_plan(sys, precision, true);
    *bytes = dmc_own_bytes(n_walk, sys->d.n_elec) + bytes_for(p, std::min(n_walk, 65535));
    return QMC_OK;
}

extern "C" int qmc_dmc_step(const qmc_system *sys, int n_walk, const qmc_walker_state *in,
                            const qmc_walker_state *out, const qmc_dmc_params *prm, double *stats, void *ws,
                            size_t ws_bytes, qmc_stream_t stream)
{
    if (!sys || !prm) return invalid("qmc_dmc_step: null argument");
    if (n_walk < 0 || n_walk > kMaxSrmcWalkers) return invalid("qmc_dmc_step: need 0 <= n_walk <= 2^24");
    if (!(prm->tau > 0.0) || !isfinite(prm->tau)) return invalid("qmc_dmc_step: tau must be positive and finite");
    if (prm->precision < QMC_PREC_F64 || prm->precision > QMC_PREC_F64_TCA4) return invalid("qmc_dmc_step: precision");
    if (n_walk == 0) return QMC_OK;
    if (!state_ok(in) || !state_ok(out) || !ws) return invalid("qmc_dmc_step: null pointer");
    if (in->R == out->R || in->drift == out->drift || in->e_loc == out->e_loc || in->status == out->status)
        return invalid("qmc_dmc_step: out may not alias in");
    const SysDev &s = sys->d;
    DmcCarve c;
    const Plan p = make_plan(sys, prm->precision, true);
    if (!dmc_carve(n_walk, s.n_elec, ws, ws_bytes, c) || bytes_for(p, 1) > c.eval_bytes) {
        set_error("qmc_dmc_step: workspace smaller than the step's arrays plus one walker's evaluation");
        return QMC_ERR_CAPACITY;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSetDevice(sys->device);
    if (e != cudaSuccess) return cuda_fail(e, "qmc_dmc_step: cudaSetDevice");
    // Eq. (1)
    e = launch_dmc_move(n_walk, s.n_elec, in->R, in->drift, prm->tau, prm->seed, prm->step, prm->step_ptr, c.R, st);
    if (e != cudaSuccess) return cuda_fail(e, "qmc_dmc_step: move launch");
    // a1..a6 at the proposed positions
    qmc_eval_out eo;
    memset(&eo, 0, sizeof eo);
    eo.logpsi = c.lp; eo.sign = c.sg; eo.drift = c.drift; eo.e_loc = c.e; eo.status = c.st;
    int rc = eval_impl(sys, n_walk, c.R, prm->precision, &eo, c.eval_ws, c.eval_bytes, st, nullptr);
    if (rc) return rc;
    // Eq. (3) with the fixed-node rule, then the reconfiguration of Sec. II.B
    e = launch_dmc_weight(n_walk, in->e_loc, in->sign, in->status, c.e, c.sg, c.st, prm->tau, prm->e_trial,
                          prm->e_trial_ptr, c.w, c.acc, st);
    if (e == cudaSuccess)
        e = launch_srmc(n_walk, c.w, prm->seed, prm->step, prm->step_ptr, c.C, c.idx, stats, c.e, in->e_loc, c.acc, st);
    if (e != cudaSuccess) return cuda_fail(e, "qmc_dmc_step: weight / reconfiguration launch");
    qmc_walker_state prop;
    prop.R = c.R; prop.drift = c.drift; prop.e_loc = c.e; prop.logpsi = c.lp; prop.sign = c.sg; prop.status = c.st;
    e = launch_dmc_gather(n_walk, s.n_elec, c.idx, c.acc, *in, prop, *out, prm->step_ptr, st);
    if (e != cudaSuccess) return cuda_fail(e, "qmc_dmc_step: gather launch");
    return QMC_OK;
}

// ---------------------------------------------------------------------------
// Mixed batch: segments of several systems, concurrent on forked streams.
namespace {

constexpr int kPoolStreams = 8;

struct StreamPool {
    int device = -1;
    cudaStream_t st[kPoolStreams] = {};
    cudaEvent_t fork = nullptr, done[kPoolStreams] = {};
};
StreamPool g_pool[kMaxDevices];

int pool_for(int dev, StreamPool **out)
{
    if (dev < 0 || dev >= kMaxDevices) return invalid("batch: device index out of range");
    StreamPool &p = g_pool[dev];
    if (p.device != dev) {
        cudaError_t e = cudaSetDevice(dev);
        for (int q = 0; q < kPoolStreams && e == cudaSuccess; ++q)
            e = cudaStreamCreateWithFlags(&p.st[q], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming);
        for (int q = 0; q < kPoolStreams && e == cudaSuccess; ++q)
            e = cudaEventCreateWithFlags(&p.done[q], cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "batch: stream pool");
        p.device = dev;
    }
    *out = &p;
    return QMC_OK;
}

int check_segments(const qmc_segment *segs, int n_seg, int precision)
{
    if (!segs || n_seg < 1) return invalid("batch: need at least one segment");
    if (precision < QMC_PREC_F64 || precision > QMC_PREC_F64_TCA4) return invalid("batch: precision");
    for (int i = 0; i < n_seg; ++i) {
        if (!segs[i].sys || segs[i].n_walk < 0) return invalid("batch: bad segment");
        if (segs[i].sys->device != segs[0].sys->device) return invalid("batch: segments on different devices");
    }
    return QMC_OK;
}

size_t seg_bytes(const qmc_segment &g, int precision)
{
    const Plan p = make_plan(g.sys, precision, g.out.dinv == nullptr);
    return al(bytes_for(p, std::max(g.n_walk, 1)));
}

}  // namespace

extern "C" int qmc_batch_workspace_size(const qmc_segment *segs, int n_seg, int precision, size_t *bytes)
{
    int rc = check_segments(segs, n_seg, precision);
    if (rc) return rc;
    if (!bytes) return invalid("qmc_batch_workspace_size: null bytes");
    size_t tot = 0;
    for (int i = 0; i < n_seg; ++i) tot += seg_bytes(segs[i], precision);
    *bytes = tot;
    return QMC_OK;
}

extern "C" int qmc_batch_eval(const qmc_segment *segs, int n_seg, int precision, void *ws, size_t ws_bytes,
                              qmc_stream_t stream)
{
    int rc = check_segments(segs, n_seg, precision);
    if (rc) return rc;
    size_t need = 0;
    for (int i = 0; i < n_seg; ++i) need += seg_bytes(segs[i], precision);
    if (need > ws_bytes) {
        set_error("qmc_batch_eval: workspace smaller than qmc_batch_workspace_size");
        return QMC_ERR_CAPACITY;
    }
    StreamPool *pool = nullptr;
    if ((rc = pool_for(segs[0].sys->device, &pool))) return rc;
    cudaStream_t main = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaEventRecord(pool->fork, main);
    if (e != cudaSuccess) return cuda_fail(e, "qmc_batch_eval: fork");
    const int nst = std::min(n_seg, kPoolStreams);
    for (int q = 0; q < nst; ++q)
        if ((e = cudaStreamWaitEvent(pool->st[q], pool->fork, 0)) != cudaSuccess)
            return cuda_fail(e, "qmc_batch_eval: fork wait");
    char *base = static_cast<char *>(ws);
    for (int i = 0; i < n_seg; ++i) {
        const size_t b = seg_bytes(segs[i], precision);
        rc = eval_impl(segs[i].sys, segs[i].n_walk, segs[i].R, precision, &segs[i].out, base, b,
                       pool->st[i % kPoolStreams], nullptr);
        if (rc) return rc;
        base += b;
    }
    for (int q = 0; q < nst; ++q) {
        if ((e = cudaEventRecord(pool->done[q], pool->st[q])) != cudaSuccess ||
            (e = cudaStreamWaitEvent(main, pool->done[q], 0)) != cudaSuccess)
            return cuda_fail(e, "qmc_batch_eval: join");
    }
    return QMC_OK;
}

struct qmc_graph {
    int device;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

extern "C" int qmc_batch_graph_create(const qmc_segment *segs, int n_seg, int precision, void *ws, size_t ws_bytes,
                                      qmc_graph **out)
{
    int rc = check_segments(segs, n_seg, precision);
    if (rc) return rc;
    if (!out) return invalid("qmc_batch_graph_create: null out");
    *out = nullptr;
    const int dev = segs[0].sys->device;
    StreamPool *pool = nullptr;
    if ((rc = pool_for(dev, &pool))) return rc;
    cudaStream_t cap = nullptr;
    cudaError_t e = cudaSetDevice(dev);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "qmc_batch_graph_create: stream");
    // first run outside capture: kernel attributes are set, tables touched
    rc = qmc_batch_eval(segs, n_seg, precision, ws, ws_bytes, reinterpret_cast<qmc_stream_t>(cap));
    if (rc == QMC_OK && (e = cudaStreamSynchronize(cap)) != cudaSuccess) rc = cuda_fail(e, "qmc_batch_graph_create");
    if (rc) { cudaStreamDestroy(cap); return rc; }
    qmc_graph *g = new qmc_graph();
    g->device = dev;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) { delete g; cudaStreamDestroy(cap); return cuda_fail(e, "qmc_batch_graph_create: capture"); }
    rc = qmc_batch_eval(segs, n_seg, precision, ws, ws_bytes, reinterpret_cast<qmc_stream_t>(cap));
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(cap, &graph);
    cudaStreamDestroy(cap);
    if (rc || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        delete g;
        return rc ? rc : cuda_fail(e, "qmc_batch_graph_create: end capture");
    }
    e = cudaGraphInstantiate(&g->exec, graph, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); delete g; return cuda_fail(e, "qmc_batch_graph_create: instantiate"); }
    g->graph = graph;
    *out = g;
    return QMC_OK;
}

extern "C" int qmc_graph_launch(qmc_graph *g, qmc_stream_t stream)
{
    if (!g) return invalid("qmc_graph_launch: null graph");
    cudaError_t e = cudaGraphLaunch(g->exec, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "qmc_graph_launch");
    return QMC_OK;
}

extern "C" int qmc_graph_free(qmc_graph *g)
{
    if (!g) return QMC_OK;
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    delete g;
    return QMC_OK;
}
