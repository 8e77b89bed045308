// Internal declarations shared by the libqmcgb translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/qmcgb.h"

namespace qmc {

constexpr int kMaxL = 4;          // highest angular momentum accepted
constexpr int kMaxPrim = 16;      // primitives per shell
constexpr int kGjPanel = 16;      // Gauss-Jordan panel width
constexpr int kMaxN = 1024;       // largest Slater matrix

// Bounded device waits of the tensor-core kernels.  limit_ns bounds each wait
// for a copy or an MMA that feeds the next step; after a wait gives up, a CTA
// waits at most kDrainNs for its own MMAs still in flight, then frees its TMEM.
// expire_w >= 0 is a test hook: the CTAs that work on that walker (index within
// the launch) wait on a flag that nothing sets instead, so their wait runs out.
constexpr unsigned long long kDrainNs = 2000000000ull;
struct WaitCfg {
    unsigned long long limit_ns = 2000000000ull;
    int expire_w = -1;
    int expire_kernels = 0;     // QMC_EXPIRE_* bits: the kernels the hook applies to
};

// Device view of a system, passed by value to kernels.
struct SysDev {
    int n_atom, n_shell, n_ao, n_up, n_dn, n_elec;
    const double *Q;        // [n_atom][3]
    const double *Z;        // [n_atom]
    const int *atom_sh0;    // [n_atom + 1] shell range of each atom
    const double *atom_R2;  // [n_atom] max of the atom's shell R2 (early exit)
    const int *sh_atom;     // [n_shell]
    const int *sh_L;
    const int *sh_nprim;
    const int *sh_pstart;
    const int *sh_ao0;      // first AO of the shell
    const double *sh_R2;    // [n_shell]
    const double *pg;       // [n_prim] exponents
    const double *pc;       // [n_prim] coefficients
    const int *ao_pow;      // [n_ao] packed nx | ny << 8 | nz << 16
    const int *ao_shell;    // [n_ao]
    const double *ao_scale; // [n_ao]
    const double *A64[2];   // [n_ao][n_s] FP64 MO coefficients per spin
    double vnn;
    // Jastrow factor e^J (off unless jas): U_ee = a r / (1 + jb_ee r), a = ja_par or ja_anti;
    // U_en = -ja_en[atom] r / (1 + jb_en[atom] r)
    int jas;
    double ja_par, ja_anti, jb_ee;
    const double *ja_en, *jb_en;   // [n_atom]
};

// Float-pair (hi + lo) copies of the basis for the float-float AO evaluation.
struct FfBasis {
    const float2 *pg, *pc;             // exponents and coefficients [n_prim]
    const float2 *sc;                  // ao_scale [n_ao]
    const float2 *Q;                   // nuclear positions [n_atom][3]
    const float2 *expj;                // exp(-j/32) for j = -12..12 (index j + 12)
};

// Exact slices for the tensor-core C1/C5 products: a value x with |x| < 2^E
// is x = 2^E (s_0 + ... + s_5 + r), s_j = q_j 2^(-7 (j + 1)), q_j integer
// (|q_0| <= 128, |q_j| <= 64 + 1 for j >= 1, so each s_j is exact in BF16), |r| < 2^-42.
constexpr int kC15Slices = 6;
constexpr int kC15SliceBits = 7;

// Split-precision copies of the MO coefficients for the mixed path, per spin.
struct MixedTables {
    const uint16_t *bhi[2], *blo[2];   // BF16 hi/lo planes [n_ao][ns_pad], ns_pad = ns rounded up to 64
    const uint16_t *hhi[2], *hlo[2];   // FP16 hi/lo planes of A * 2^a_exp[spin], same layout
    const float2 *ff[2];               // float-float (hi, lo) plane [n_ao][ns32], zero beyond ns
    int ns32[2];                       // ns rounded up to 32
    const float *colmax[2];            // max over AOs of |A[mu][k]| per MO column k [ns32], zero beyond ns
    const uint16_t *slice[2];          // BF16 slices s_j of A[mu][k] 2^-F_k: [kC15Slices][n_ao][ns_pad]
    const int *fexp[2];                // F_k per MO column [ns_pad] (|A[.][k]| < 2^F_k)
    const uint16_t *rslice[2];         // BF16 slices of A[mu][k] 2^-G_mu (per-AO-row exponents, for the
                                       // C-free product v = D^-1 A^T): [kC15Slices][n_ao][ns_pad]
    const int *gexp[2];                // G_mu per AO row [n_ao] (|A[mu][.]| < 2^G_mu)
    int ns_pad[2];
    int a_exp[2];                      // FP16 planes hold A * 2^a_exp
    int b_exp;                         // FP16 path: AO gradients enter scaled by 2^b_exp
    int mask_words;                    // 32-bit words of a per-electron shell bitmask
    const float *pgf, *pcf;            // FP32 copies of exponents and coefficients [n_prim]
    const float *scf;                  // FP32 copy of ao_scale [n_ao]
    const float *Qhi, *Qlo;            // nuclear positions as float pairs [n_atom][3]
    const float *atom_R2f, *sh_R2f;    // screening radii rounded to float [n_atom], [n_shell]
    FfBasis ffb;
};

struct TcTables {                      // what the tensor-core kernel reads, one precision mode
    const uint16_t *hi[2], *lo[2];
    int ns_pad[2];
    int f16;                           // 1: FP16 operands, 0: BF16
    float out_scale[2][3];             // multiply accumulator (spin, gradient component) by this (power of 2)
    float in_scale[3];                 // multiply AO gradient component l by this before the split
    const float *pgf, *pcf, *scf, *Qhi, *Qlo;
};

// Per-matrix parameters for the Gauss-Jordan kernel (one entry per spin).
struct GjJob {
    double *X;          // first matrix
    long long x_stride; // elements between consecutive matrices
    double *Dinv;
    long long d_stride;
    double *logabs;     // may be null
    long long la_stride;
    double *sign;       // may be null
    uint32_t *flag;     // may be null: OR-ed with flag_bit on exact zero pivot
    uint32_t flag_bit;
    int n;
    int count;
    float2 *work;       // float-float elimination: float-pair work matrices (x_stride apart)
    uint8_t *redo;      // float-float: set to 1 for matrices the FP64 kernel must recompute
    long long redo_stride;
    int only_redo;      // FP64 kernel: process only matrices with redo[m] == 1 (flagged, not recomputed yet)
};

void set_error(const std::string &msg);
int cuda_fail(cudaError_t e, const char *where);

// kernels (launchers); all return a cudaError_t from the launch
cudaError_t launch_contract_f64(const SysDev &s, int nw, const double *R, double *X, double *Cd,
                                cudaStream_t st);
cudaError_t launch_screen_ao(const SysDev &s, int nw, const double *R, int cap, int32_t *cnt,
                             int32_t *idx, double *B, cudaStream_t st);
cudaError_t launch_gj(const GjJob *jobs, int n_jobs, cudaStream_t st, int nb);
// Multi-CTA FP64 recomputation of up to kRedoMax flagged matrices (redo 1 -> 2).
constexpr int kRedoMax = 256;
size_t redo_scratch_bytes(int nmax);
cudaError_t launch_gj_redo(const GjJob *jobs, int n_jobs, void *scratch, cudaStream_t st, int nb, const SysDev *s,
                           const double *R, const int *e_off);
cudaError_t launch_gj_ff(const GjJob *jobs, int n_jobs, cudaStream_t st, int nb, double kappa_max);
// Where the gradient (C2..C4) and Laplacian (C5) matrices of a walker chunk live:
// component c of spin s, electron row ei: base + w*wstride + (s ? ncomp*n_up^2 : 0) + c*ns^2 + ei*ns
struct CView {
    const void *g;      // gradients, FP32 if g_f32 else FP64
    int g_f32;
    size_t g_wstride;
    int g_ncomp;
    const double *l;    // Laplacian, FP64, component l_comp of its block
    size_t l_wstride;
    int l_ncomp;
    int l_comp;
    const double *vd;   // C-free variant: drift and Laplacian per electron [W][N][4] (the dots are done)
};

cudaError_t launch_drift_energy(const SysDev &s, int nw, const double *R, const double *Dinv, const CView &cv,
                                const double *logabs2, const double *sign2, const uint32_t *sing,
                                const qmc_eval_out &o, int w_off, cudaStream_t st, const float2 *Q2);
cudaError_t launch_shell_mask(const SysDev &s, const MixedTables &mt, int nw, const double *R, int mw,
                              uint32_t *masks, cudaStream_t st);
cudaError_t launch_c15_ff(const SysDev &s, const FfBasis &fb, int nw, const double *R, const uint32_t *masks,
                          int mw, const float2 *const *A, const int *ns32, const float *const *colmax,
                          double *X, double *L5, cudaStream_t st, int walkers_per_cta);
bool c15tc_fits(const SysDev &s, int mw);
size_t c15tc_bytes(const SysDev &s, int nw);
cudaError_t launch_c15_tc(const SysDev &s, const FfBasis &fb, const MixedTables &mt, const TcTables &tt, int nw,
                          const double *R, const uint32_t *masks, int mw, double *X, double *L5, float *Cg,
                          uint32_t *wstatus, void *scratch, cudaStream_t st, const WaitCfg &wc,
                          bool c1_only = false);
// C-free variant: drift and Laplacian from v = D^-1 A^T (k_vdrift.cu)
bool vdrift_fits(const SysDev &s);
size_t vdrift_bytes(const SysDev &s, int nw);
cudaError_t launch_vdrift(const SysDev &s, const FfBasis &fb, const MixedTables &mt, int nw, const double *R,
                          const uint32_t *masks, int mw, const double *Dinv, double *vd, uint32_t *wstatus,
                          void *scratch, cudaStream_t st, const WaitCfg &wc);
cudaError_t launch_tc_contract(const SysDev &s, int nw, const double *R, const uint32_t *masks, int mw,
                               const TcTables &tt, float *Cg, uint32_t *wstatus, cudaStream_t st, const WaitCfg &wc);
cudaError_t launch_widen(const float *src, size_t spitch, double *dst, size_t dpitch, size_t width, int rows,
                         cudaStream_t st);
// AO blocks of the tensor-core adjoint: runs of consecutive whole atoms with at
// most nb AOs (nb = TMEM columns per MO tile).
struct BwBlocks {
    int nblk = 0, nb = 0;
    const int *ao0 = nullptr, *sh0 = nullptr;   // [nblk + 1] first AO / first shell of each block
};
constexpr int kBwtChunk = 512;                  // walkers per pass of the tensor-core adjoint
int bwtc_block_width(int nmax);
size_t bwtc_bytes(const SysDev &s, int mw, int nw, int wb);
cudaError_t launch_backward_tc(const SysDev &s, const MixedTables &mt, const BwBlocks &bb, int wb, int nw,
                               const double *R,
                               const double *dinv, const double *g, double *dA_up, double *dA_dn, void *ws,
                               size_t ws_bytes, cudaStream_t st, const WaitCfg &wc);
// a4 of the mixed path with the panel updates on the tensor cores
// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against the
// driver library): a rank-d map of 8- or 16-bit elements, row-major, boxes `box`,
// the given swizzle, zero fill outside the tensor.  strides[] are the byte strides of
// dimensions 1..rank-1 (multiples of 16).
cudaError_t tmap_encode(CUtensorMap *m, CUtensorMapDataType dt, int rank, const void *addr, const uint64_t *dims,
                        const uint64_t *strides, const uint32_t *box, CUtensorMapSwizzle swz);

bool gjtc_fits(int nmax);
size_t gjtc_bytes(int n_up, int n_dn, int nw);
cudaError_t launch_gj_tc(const GjJob *jobs, int n_jobs, void *scratch, cudaStream_t st, double kappa_max,
                         const WaitCfg &wc);
cudaError_t launch_backward_f64(const SysDev &s, int nw, const double *R, const double *dinv,
                                const double *g, double *dA_up, double *dA_dn, cudaStream_t st,
                                int max_ao_per_atom);

// Multi-determinant expansion (k_multidet.cu)
constexpr int kMaxDets = 64;
cudaError_t launch_multidet_combine(int nw, int N, int K, const double *coef, const double *lp, const double *sg,
                                    const double *dr, const double *el, const double *ep, const uint32_t *st,
                                    const qmc_eval_out &o, cudaStream_t stream);

// Monte Carlo step (k_dmc.cu)
cudaError_t launch_dmc_move(int nw, int n_elec, const double *R, const double *drift, double tau, uint64_t seed,
                            uint64_t step, const uint64_t *step_ptr, double *Rn, cudaStream_t st);
cudaError_t launch_dmc_weight(int nw, const double *e_old, const double *s_old, const uint32_t *st_old,
                              const double *e_new, const double *s_new, const uint32_t *st_new, double tau,
                              double e_trial, const double *e_trial_ptr, double *weight, uint32_t *accept,
                              cudaStream_t st);
cudaError_t launch_srmc(int nw, const double *weight, uint64_t seed, uint64_t step, const uint64_t *step_ptr,
                        unsigned long long *C, int *idx, double *stats, const double *e_new, const double *e_old,
                        const uint32_t *accept, cudaStream_t st);
cudaError_t launch_dmc_gather(int nw, int n_elec, const int *idx, const uint32_t *accept, const qmc_walker_state &old,
                              const qmc_walker_state &prop, const qmc_walker_state &out, uint64_t *step_ptr,
                              cudaStream_t st);

}  // namespace qmc

struct qmc_system {
    int device;
    qmc_tiles tiles;                  // tile choices (autotuned or default)
    qmc::SysDev d;
    std::vector<void *> allocs;     // device allocations owned by the system
    std::vector<double> R2_host;
    qmc::MixedTables mixed;
    int max_shell_per_atom;
    qmc::BwBlocks bw;                 // AO blocks of the tensor-core adjoint
    void *mo_dev = nullptr;           // device tables derived from the MO coefficients
    size_t mo_bytes = 0;
    int a_dtype = 0;
    uint32_t crc_prefix = 0;          // CRC-32 register after the basis arrays (before A_up)
    uint32_t crc = 0;                 // CRC-32 key of the critical data
    uint32_t crc_nojas = 0;           // the key without the Jastrow parameters
    double eps = 0.0;
};
