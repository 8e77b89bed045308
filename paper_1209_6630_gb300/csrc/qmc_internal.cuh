// Internal declarations shared by the libqmcgb translation units.
#pragma once

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
};

// Split-precision tables of the mixed path (per spin).
struct MixedTables {
    // A^T split planes, K-major bf16: [plane][n_s_pad][n_ao_pad]
    uint16_t *At[2];
    int n_s_pad[2];
    int n_ao_pad;
    int n_planes;
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
};

void set_error(const std::string &msg);
int cuda_fail(cudaError_t e, const char *where);

// kernels (launchers); all return a cudaError_t from the launch
cudaError_t launch_contract_f64(const SysDev &s, int nw, const double *R, double *X, double *Cd,
                                cudaStream_t st);
cudaError_t launch_screen_ao(const SysDev &s, int nw, const double *R, int cap, int32_t *cnt,
                             int32_t *idx, double *B, cudaStream_t st);
cudaError_t launch_gj(const GjJob *jobs, int n_jobs, cudaStream_t st);
cudaError_t launch_drift_energy(const SysDev &s, int nw, const double *R, const double *Dinv,
                                const double *Cd, int cd_is_f32, const double *logabs2,
                                const double *sign2, const uint32_t *sing, const qmc_eval_out &o,
                                int w_off, cudaStream_t st);
cudaError_t launch_backward_f64(const SysDev &s, int nw, const double *R, const double *dinv,
                                const double *g, double *dA_up, double *dA_dn, cudaStream_t st,
                                int max_ao_per_atom);

}  // namespace qmc

struct qmc_system {
    int device;
    qmc::SysDev d;
    std::vector<void *> allocs;     // device allocations owned by the system
    std::vector<double> R2_host;
    qmc::MixedTables mixed;
    int max_shell_per_atom;
};
