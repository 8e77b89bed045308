// Host side of libqmcgb: system loading, workspace planning and the C ABI
// entry points declared in include/qmcgb.h.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

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
    std::vector<double> A64[2];
    for (int spin = 0; spin < 2; ++spin) {
        const int ns = spin ? nd : nu;
        const void *src = spin ? d->A_dn : d->A_up;
        A64[spin].resize((size_t)nao * ns);
        for (size_t q = 0; q < (size_t)nao * ns; ++q)
            A64[spin][q] = d->a_dtype == QMC_DTYPE_F64 ? static_cast<const double *>(src)[q]
                                                       : (double) static_cast<const float *>(src)[q];
    }

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
    const size_t oA0 = b.add(A64[0].data(), sizeof(double) * A64[0].size());
    const size_t oA1 = b.add(A64[1].data(), sizeof(double) * A64[1].size());

    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) { delete sys; return cuda_fail(e, "qmc_system_load: cudaSetDevice"); }
    char *dev = nullptr;
    e = cudaMalloc(&dev, b.host.size());
    if (e != cudaSuccess) { delete sys; return cuda_fail(e, "qmc_system_load: cudaMalloc"); }
    sys->allocs.push_back(dev);
    e = cudaMemcpy(dev, b.host.data(), b.host.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { qmc_system_free(sys); return cuda_fail(e, "qmc_system_load: cudaMemcpy"); }

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
    s.A64[0] = reinterpret_cast<const double *>(dev + oA0);
    s.A64[1] = reinterpret_cast<const double *>(dev + oA1);
    s.vnn = vnn;
    memset(&sys->mixed, 0, sizeof(sys->mixed));
    *out = sys;
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
namespace {

struct Plan {
    size_t msz;        // n_up^2 + n_dn^2
    size_t per_walker; // bytes
    size_t oX, oCd, oD, oLa, oSg, oSt;
};

size_t al(size_t x) { return (x + 255) & ~size_t(255); }

Plan make_plan(const qmc_system *sys, int precision, bool need_dinv)
{
    Plan p;
    p.msz = (size_t)sys->d.n_up * sys->d.n_up + (size_t)sys->d.n_dn * sys->d.n_dn;
    const size_t cd_elem = precision == QMC_PREC_F64 ? 8 : 4;
    size_t o = 0;
    p.oX = o; o += p.msz * 8;
    p.oCd = o; o += 4 * p.msz * cd_elem;
    p.oD = o; o += need_dinv ? p.msz * 8 : 0;
    p.oLa = o; o += 16;
    p.oSg = o; o += 16;
    p.oSt = o; o += 4;
    p.per_walker = o;
    return p;
}

struct Carve {
    double *X; void *Cd; double *D; double *la; double *sg; uint32_t *st;
};

// Arrays for `nw` walkers laid out array by array inside ws.
bool carve(const Plan &p, int nw, void *ws, size_t ws_bytes, Carve &c)
{
    char *b = static_cast<char *>(ws);
    size_t o = 0;
    auto take = [&](size_t bytes) { char *r = b + o; o = al(o + bytes); return r; };
    c.X = reinterpret_cast<double *>(take(p.msz * 8 * nw));
    c.Cd = take((p.oD - p.oCd) * nw);
    c.D = (p.oLa - p.oD) ? reinterpret_cast<double *>(take(p.msz * 8 * nw)) : nullptr;
    c.la = reinterpret_cast<double *>(take(16 * (size_t)nw));
    c.sg = reinterpret_cast<double *>(take(16 * (size_t)nw));
    c.st = reinterpret_cast<uint32_t *>(take(4 * (size_t)nw));
    return o <= ws_bytes;
}

size_t bytes_for(const Plan &p, int nw)
{
    return al(p.msz * 8 * nw) + al((p.oD - p.oCd) * nw) + ((p.oLa - p.oD) ? al(p.msz * 8 * nw) : 0) +
           al(16 * (size_t)nw) * 2 + al(4 * (size_t)nw);
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

}  // namespace

extern "C" int qmc_workspace_size(const qmc_system *sys, int n_walk, int precision, size_t *bytes)
{
    if (!sys || !bytes || n_walk < 0) return invalid("qmc_workspace_size: bad argument");
    if (precision != QMC_PREC_F64 && precision != QMC_PREC_MIXED) return invalid("qmc_workspace_size: precision");
    const Plan p = make_plan(sys, precision, true);
    *bytes = bytes_for(p, std::min(n_walk, 65535));
    return QMC_OK;
}

extern "C" int qmc_walkers_eval(const qmc_system *sys, int n_walk, const double *R, int precision,
                                const qmc_eval_out *out, void *ws, size_t ws_bytes, qmc_stream_t stream)
{
    if (!sys || !out) return invalid("qmc_walkers_eval: null argument");
    if (n_walk < 0) return invalid("qmc_walkers_eval: n_walk < 0");
    if (n_walk == 0) return QMC_OK;
    if (!R || !out->logpsi || !out->sign || !out->drift || !out->e_loc || !out->status)
        return invalid("qmc_walkers_eval: null required pointer");
    if (precision != QMC_PREC_F64) return invalid("qmc_walkers_eval: precision not available in this build");
    const Plan p = make_plan(sys, precision, out->dinv == nullptr);
    const int chunk = chunk_walkers(p, n_walk, ws_bytes);
    if (chunk < 1) {
        set_error("qmc_walkers_eval: workspace smaller than one walker");
        return QMC_ERR_CAPACITY;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const SysDev &s = sys->d;
    cudaError_t e = cudaSetDevice(sys->device);
    if (e != cudaSuccess) return cuda_fail(e, "qmc_walkers_eval: cudaSetDevice");
    for (int w0 = 0; w0 < n_walk; w0 += chunk) {
        const int nw = std::min(chunk, n_walk - w0);
        Carve c;
        carve(p, nw, ws, ws_bytes, c);
        const double *Rc = R + (size_t)w0 * s.n_elec * 3;
        double *Dinv = out->dinv ? out->dinv + (size_t)w0 * p.msz : c.D;
        e = cudaMemsetAsync(c.st, 0, 4 * (size_t)nw, st);
        if (e != cudaSuccess) return cuda_fail(e, "qmc_walkers_eval: memset");
        e = launch_contract_f64(s, nw, Rc, c.X, static_cast<double *>(c.Cd), st);
        if (e != cudaSuccess) return cuda_fail(e, "qmc_walkers_eval: contraction launch");
        GjJob jobs[2];
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
        }
        e = launch_gj(jobs, nj, st);
        if (e != cudaSuccess) return cuda_fail(e, "qmc_walkers_eval: Gauss-Jordan launch");
        e = launch_drift_energy(s, nw, Rc, Dinv, static_cast<double *>(c.Cd), precision != QMC_PREC_F64, c.la,
                                c.sg, c.st, *out, w0, st);
        if (e != cudaSuccess) return cuda_fail(e, "qmc_walkers_eval: energy launch");
    }
    return QMC_OK;
}

extern "C" int qmc_slater_matrices(const qmc_system *sys, int n_walk, const double *R, int precision, double *C,
                                   void *ws, size_t ws_bytes, qmc_stream_t stream)
{
    if (!sys || (n_walk > 0 && (!R || !C))) return invalid("qmc_slater_matrices: null argument");
    if (n_walk < 0) return invalid("qmc_slater_matrices: n_walk < 0");
    if (precision != QMC_PREC_F64) return invalid("qmc_slater_matrices: precision not available in this build");
    if (n_walk == 0) return QMC_OK;
    const Plan p = make_plan(sys, precision, false);
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
        double *Cd = static_cast<double *>(c.Cd);
        e = launch_contract_f64(s, nw, Rc, c.X, Cd, st);
        if (e != cudaSuccess) return cuda_fail(e, "qmc_slater_matrices: contraction launch");
        char *o = reinterpret_cast<char *>(C + (size_t)w0 * 5 * p.msz);
        // per walker: [C1 up][C2..C5 up][C1 dn][C2..C5 dn]
        struct { const double *src; size_t spitch, width, dst_off; } cp[4] = {
            {c.X, p.msz * 8, nu2 * 8, 0},
            {Cd, 4 * p.msz * 8, 4 * nu2 * 8, nu2 * 8},
            {c.X + nu2, p.msz * 8, nd2 * 8, 5 * nu2 * 8},
            {Cd + 4 * nu2, 4 * p.msz * 8, 4 * nd2 * 8, 6 * nu2 * 8},
        };
        for (auto &q : cp) {
            if (q.width == 0) continue;
            e = cudaMemcpy2DAsync(o + q.dst_off, opitch, q.src, q.spitch, q.width, nw, cudaMemcpyDeviceToDevice, st);
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
    GjJob j;
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
    cudaError_t e = launch_gj(&j, 1, st);
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
