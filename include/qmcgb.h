/*
 * qmcgb.h -- C ABI of libqmcgb: batched all-electron walker evaluation with
 * Slater matrices built from localized atomic Gaussians (arXiv:1209.6630,
 * "Quantum Monte Carlo for large chemical systems: implementing efficient
 * strategies for petascale platforms and beyond"), on one NVIDIA GB300
 * (sm_103a).
 *
 * What one walker evaluation computes (the paper's hot spot, Sec. II.C):
 *   for a walker R = (r_1..r_N) and a single-determinant trial function
 *   Psi = Det_up * Det_dn (no Jastrow; the benchmarks of Sec. III are
 *   Hartree-Fock wave functions):
 *     a1  screening: AO chi_mu is zero for electron e where its radial part
 *         g < eps (Sec. III; radius test d2 < R2_shell, atomic early exit)
 *     a2  AO values, gradients and Laplacians (Sec. II.C, AO form)
 *     a3  the five products C_l = A B_l, l=1..5 (Sec. III, Eq. "abc")
 *     a4  log|det|, sign and inverse of each spin's Slater matrix
 *         (Sec. II.C; inversion step of Sec. IV.B)
 *     a5  drift b = grad Psi / Psi (Eq. 2) and kinetic energy from D^-1 and
 *         the Laplacian matrix (Sec. II.C vector products)
 *     a6  local energy E_L = H Psi / Psi (Eq. 4) with the all-electron
 *         Coulomb Hamiltonian: T + V_en + V_ee + V_nn
 *     a7  adjoint d log|Psi| / dA for parameter optimisation
 *
 * Conventions (every entry point):
 *   - Return value: QMC_OK (0) or a negative QMC_ERR_* code; the message of
 *     the last failing call on this thread is in qmc_last_error().
 *   - "device" pointers are CUDA device memory of the system's device, owned
 *     by the caller; "host" pointers are ordinary host memory, only read
 *     during the call.  Device work is queued on `stream` (NULL = legacy
 *     default stream) and is asynchronous unless stated otherwise.
 *   - A numerical failure of one walker (exactly singular Slater matrix,
 *     non-finite input or result) is not a call error: it sets bits in that
 *     walker's status word and the rest of the batch is valid.
 *   - Layouts are row-major.  Electrons 0..n_up-1 are spin up, the rest
 *     spin down (Sec. II.C: the first N_up electrons enter Det_up).
 *   - There is no CPU fallback: without a usable GB300 every call fails.
 */
#ifndef QMCGB_H
#define QMCGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *qmc_stream_t;   /* the same handle as cudaStream_t */
typedef struct qmc_system qmc_system;       /* opaque, device-resident system */

enum {
    QMC_OK = 0,
    QMC_ERR_INVALID = -1,   /* bad argument, size or layout */
    QMC_ERR_CUDA = -2,      /* a CUDA runtime/driver call failed */
    QMC_ERR_TIMEOUT = -3,   /* a bounded device wait gave up */
    QMC_ERR_CAPACITY = -4,  /* workspace too small / size above a kernel limit */
    QMC_ERR_NOMEM = -5      /* the library could not allocate its own tables */
};

/* per-walker status bits */
enum {
    QMC_STATUS_SINGULAR_UP = 1u,   /* exact zero pivot in Det_up: log|Psi| = -inf, sign = 0 */
    QMC_STATUS_SINGULAR_DN = 2u,
    QMC_STATUS_NONFINITE = 4u,     /* non-finite coordinate or result */
    QMC_STATUS_TIMEOUT = 8u        /* a bounded wait inside a tensor-core kernel gave up
                                      for this walker's tile: its results are invalid */
};

/* arithmetic of an evaluation (the screening decisions a1 are the exact FP64
 * ones in both) */
enum {
    QMC_PREC_F64 = 0,        /* plain FP64 path: AO values, products, LU, energies in FP64 */
    QMC_PREC_MIXED = 1,      /* C1 (the Slater matrix) and C5 (its Laplacian) per
                                qmc_tiles.c15_mode (tcgen05 MMAs on exact BF16 slices of
                                float-float AO values and of A, or float-float products);
                                C2..C4 (gradient matrices) on the tcgen05 tensor cores from
                                FP16 hi/lo split operands (3 products, FP32 accumulation,
                                exact power-of-two scaling); a4 per qmc_tiles.a4_mode
                                (float-float Gauss-Jordan, alone or with its rank-32 updates
                                on the tensor cores, with FP64 recomputation near nodal
                                surfaces; or FP64); drift dots in FP32 and the Laplacian dot
                                in FP64, Coulomb sums in float-float, results in FP64 */
    QMC_PREC_MIXED_BF16 = 2, /* as QMC_PREC_MIXED with BF16 hi/lo splits for C2..C4 */
    QMC_PREC_F64_TCA4 = 3    /* the plain FP64 path (FP64 AO values, products and energies)
                                with a4 by the tensor-core Gauss-Jordan of the mixed path
                                (float-float panels, rank-32 updates from exact BF16 slices;
                                the float-float elimination where that kernel does not fit)
                                and the FP64 elimination (one CTA per matrix, the FP64
                                C1 kept) of every matrix whose kappa_inf exceeds
                                qmc_tiles.f64_kappa_max: a cheaper FP64-accurate a4
                                (Sec. IV.B inversion step; Table 2 caption: the inversion in
                                double precision) */
};

enum { QMC_DTYPE_F64 = 0, QMC_DTYPE_F32 = 1 };

/*
 * System description, host memory.  Sec. II.C: MOs phi_k = sum_mu a_{k mu}
 * chi_mu (Eq. "mo"); Cartesian Gaussian AOs chi_mu(r) = scale_mu
 * (x-Qx)^nx (y-Qy)^ny (z-Qz)^nz g_s(r), g_s(r) = sum_p c_p exp(-gamma_p |r-Q|^2)
 * (Eq. "Gaussian").  AOs must be stored shell by shell (each shell's
 * Cartesian components contiguous) and shells atom by atom.
 */
typedef struct {
    int n_atom;
    const double *Z;             /* [n_atom] nuclear charges */
    const double *Q;             /* [n_atom][3] positions (bohr) */
    int n_shell;
    const int32_t *shell_atom;   /* [n_shell] non-decreasing */
    const int32_t *shell_L;      /* [n_shell] angular momentum 0..4 */
    const int32_t *shell_nprim;  /* [n_shell] 1..16 primitives */
    const int32_t *shell_pstart; /* [n_shell] offset into prim_* */
    int n_prim;
    const double *prim_gamma;    /* [n_prim] exponents > 0 */
    const double *prim_coef;     /* [n_prim] contraction coefficients (> 0 for
                                    the radius search to be meaningful) */
    int n_ao;
    const int32_t *ao_shell;     /* [n_ao] */
    const int32_t *ao_pow;       /* [n_ao][3] (nx, ny, nz), nx+ny+nz = L */
    const double *ao_scale;      /* [n_ao] per-component normalisation factor */
    int n_up, n_dn;              /* electrons per spin = MOs per determinant */
    int a_dtype;                 /* QMC_DTYPE_F64 or QMC_DTYPE_F32 */
    const void *A_up;            /* [n_ao][n_up] MO coefficients, row = AO */
    const void *A_dn;            /* [n_ao][n_dn] */
    double eps;                  /* screening threshold on g (paper: 1e-8) */
    uint32_t crc32;              /* CRC-32 key of the critical data (Sec. V.C, error
                                    checking): the CRC-32 of ISO 3309 / ITU-T V.42 (the
                                    one zlib computes; reflected polynomial 0xEDB88320,
                                    initial value and final XOR 0xFFFFFFFF) over the bytes
                                    of Z, Q, shell_atom, shell_L, shell_nprim,
                                    shell_pstart, prim_gamma, prim_coef, ao_shell,
                                    ao_pow, ao_scale, A_up, A_dn (in this order, as
                                    stored in these arrays) and then eps (8 bytes,
                                    IEEE binary64, host byte order) */
} qmc_system_desc;

/*
 * qmc_system_load -- copy a system to `device` and prepare it (Sec. III).
 * Computes, on the host, each shell's screening radius R2_s = the smallest
 * non-negative double x with g_s(x) < eps (g evaluated at squared distance x;
 * bisection on the IEEE bit patterns of non-negative doubles), each atom's
 * radius (max over its shells, the paper's early exit), V_nn, and the
 * device tables (FP64 A and the split planes the mixed path reads).
 * The CRC-32 of the description is computed first (Sec. V.C: the key checks
 * that the input data reached the computing node intact); if it differs from
 * desc->crc32 nothing is loaded and the call returns QMC_ERR_INVALID with a
 * message giving both values.
 * The library owns the returned system until qmc_system_free.  Blocking.
 */
int qmc_system_load(const qmc_system_desc *desc, int device, qmc_system **out);
int qmc_system_free(qmc_system *sys);

/* The CRC-32 key of a loaded system's critical data (as checked at load;
 * qmc_system_set_mo recomputes it over the new coefficients; with a Jastrow
 * factor set, the key continues over its parameters: a_par, a_anti, b_ee as
 * three doubles, then a_en[], then b_en[]). */
int qmc_system_crc32(const qmc_system *sys, uint32_t *crc);

/*
 * Jastrow factor (Sec. II.C: Psi_T = e^J Det_up Det_dn, the Jastrow of the
 * trial-function formula with its e-n and e-e terms; the paper leaves the
 * functions U open, this library takes the Pade form):
 *   J = sum_{i<j} a r_ij / (1 + b_ee r_ij) - sum_{i,atoms} a_en[at] r / (1 + b_en[at] r),
 *   a = a_par for two electrons of the same spin, a_anti otherwise
 *   (a_anti = 1/2, a_par = 1/4 satisfy the electron-electron cusp conditions).
 * With the factor on, log|Psi| includes J (logabs stays the determinants'),
 * the drift gains grad J and the kinetic term lap J + |grad J|^2 +
 * 2 grad J . grad Det / Det; the adjoint d log|Psi| / dA is unchanged (J does
 * not depend on A).  The Jastrow sums run in FP64 in every precision mode
 * (O(N^2) per walker).  Off after qmc_system_load and after
 * qmc_system_set_mo.  enabled = 0 (or j == NULL) switches it off.
 * Blocking: synchronises the device first.  a_en, b_en: host [n_atom];
 * b_ee, b_en >= 0.
 */
typedef struct {
    int enabled;
    double a_par, a_anti, b_ee;
    const double *a_en;
    const double *b_en;
} qmc_jastrow;
int qmc_system_set_jastrow(qmc_system *sys, const qmc_jastrow *j);

/*
 * qmc_system_set_mo -- replace the MO coefficients a_{k mu} of a loaded
 * system (Eq. "mo"), e.g. between the steps of a parameter optimisation
 * driven by qmc_logpsi_backward.  A_up [n_ao][n_up], A_dn [n_ao][n_dn] host
 * arrays of a_dtype.  Rebuilds the library's device copies (FP64 and the
 * split planes of the mixed path) in place.  Blocking: it synchronises the
 * device first, so no evaluation still reads the old coefficients.  The
 * system's CRC-32 key (qmc_system_crc32) is recomputed over the new ones.
 */
int qmc_system_set_mo(qmc_system *sys, int a_dtype, const void *A_up, const void *A_dn);

/*
 * Tile and arithmetic choices of a system's kernels (set by the autotuner or
 * by hand).
 *   gj_panel           Gauss-Jordan panel width: 8, 16 or 32 columns (shared
 *                      memory n*gj_panel doubles per matrix; wider = fewer
 *                      sweeps over the matrix, fewer CTAs per SM)
 *   c15_walkers        walkers per CTA in the mixed path's C1/C5 kernel: 2 or 4
 *                      (more = fewer reads of the MO coefficients, more registers)
 *   a4_mode            a4 arithmetic of the mixed paths (the FP64 path always
 *                      uses FP64): QMC_A4_FP64, or QMC_A4_FLOAT_FLOAT = the same
 *                      Gauss-Jordan elimination on float pairs (~48-bit
 *                      significand, FP32 pipes) whose matrices with
 *                      kappa_inf = ||X||_inf ||X^-1||_inf above a4_kappa_max (near a
 *                      nodal surface), with a zero pivot or a non-finite result
 *                      are recomputed in FP64 -- their C1 from the positions
 *                      (FP64 AO values and products) and then the elimination,
 *                      since there log|det| amplifies the mixed C1's ~2^-40 error
 *                      by kappa; or QMC_A4_TENSOR = the same elimination and
 *                      recomputation with panels of 32 columns whose rank-32
 *                      updates run on the tcgen05 tensor cores (panel and pivot
 *                      rows in six exact BF16 slices, per-row / per-column
 *                      power-of-two scaling, four FP32 accumulators added to
 *                      the float-pair matrix; at most 880 electrons per spin)
 *   a4_kappa_max       that threshold (> 0)
 *   c15_mode           arithmetic of C1/C5 on the mixed paths:
 *                      QMC_C15_FLOAT_FLOAT = float-float products on the FP32
 *                      pipes; QMC_C15_TENSOR = tcgen05 BF16 MMAs on exact 7-bit
 *                      slices of both operands (six each, per-row / per-column
 *                      power-of-two scaling, four FP32 accumulators per output,
 *                      ~2^-40 normwise), with a staging buffer in the workspace;
 *                      QMC_C15_CFREE = the "C-free" variant: only C1 is formed (as
 *                      in QMC_C15_TENSOR), and after a4 the drift and Laplacian
 *                      come from v_e = D^-1[e,:] A^T (Sec. II.C vector products with
 *                      the MO expansion Eq. (mo)): drift_e = sum_mu v_e,mu grad chi_mu,
 *                      lap_e = sum_mu v_e,mu lap chi_mu over e's active AOs, v on the
 *                      tcgen05 tensor cores from exact BF16 slices of D^-1 and A
 *                      (as for C1), the AO derivatives evaluated in the epilogue
 *                      (gradient FP32, Laplacian float-float); C2..C5 are never
 *                      stored (qmc_slater_matrices still returns all five, formed
 *                      as in QMC_C15_TENSOR)
 *   bw_walkers         walkers per CTA of the tensor-core adjoint
 *                      (qmc_logpsi_backward_ex, QMC_PREC_MIXED): 2, 4, 8, 16 or
 *                      32.  A CTA's FP32 accumulators sum over its walkers'
 *                      pairs only and the CTAs' partials are added in FP64:
 *                      fewer walkers = shorter FP32 sums (smaller rounding
 *                      error), more partials written and read
 *   wait_s             limit, in seconds, of each bounded device wait of the
 *                      tcgen05 kernels for the copies and MMAs that feed their
 *                      next step (1e-6 .. 60).  A wait that runs out does not
 *                      hang the call: the C1..C5 kernels set QMC_STATUS_TIMEOUT
 *                      on the walkers of their tile of 128, the tensor-core a4
 *                      hands its matrix to the FP64 recomputation (the result
 *                      stays correct), the tensor-core adjoint leaves NaN in
 *                      the rows of dA its CTA owned.  After such a wait the CTA
 *                      waits at most 2 s more for its own MMAs, then frees its
 *                      tensor memory and returns.  (The paper's principle for
 *                      failures, Sec. V: lose only the affected block of work.)
 *   expire_walker      test hook, -1 = off.  For w >= 0 the tcgen05 kernels that
 *                      work on walker w (index within the call) make one of
 *                      their waits run out deliberately: it waits wait_s on a
 *                      flag that nothing sets.  C1..C5: the C1 CTA of electron 0
 *                      and MO tile 0 of w's walker tile; a4 (tensor mode): the
 *                      first update CTA of w's spin-up and spin-down matrices;
 *                      adjoint: the spin-up CTAs of w's block of bw_walkers.
 *   expire_kernels     which kernels the hook applies to: bits QMC_EXPIRE_C15
 *                      (1), QMC_EXPIRE_A4 (2), QMC_EXPIRE_ADJOINT (4).
 *   f64_kappa_max      QMC_PREC_F64_TCA4: matrices with kappa_inf above this are
 *                      recomputed in FP64 (> 0)
 * Defaults after qmc_system_load: gj_panel = 16 (8 if an electron count
 * exceeds 640), c15_walkers = 4, a4_mode = QMC_A4_FLOAT_FLOAT (QMC_A4_TENSOR
 * from 512 electrons of one spin on, where it fits the panel kernel),
 * a4_kappa_max = 1e8 (1e7 up to 256 electrons of one spin),
 * c15_mode = QMC_C15_CFREE where the system fits the tensor-core kernels
 * (at most 1024 electrons per spin, 8192 shells, ~7500 AOs; the C-free
 * kernel: ~36000 AOs), else QMC_C15_FLOAT_FLOAT, bw_walkers = 8, wait_s = 2, expire_walker = -1,
 * expire_kernels = 7, f64_kappa_max = 1e6 (1, i.e. every matrix in FP64, up to 256
 * electrons of one spin).
 * qmc_system_set_tiles returns QMC_ERR_INVALID for
 * other values (or a tensor mode that does not fit) and keeps the previous
 * choice.
 */
enum { QMC_A4_FP64 = 0, QMC_A4_FLOAT_FLOAT = 1, QMC_A4_TENSOR = 2 };
enum { QMC_C15_FLOAT_FLOAT = 0, QMC_C15_TENSOR = 1, QMC_C15_CFREE = 2 };
enum { QMC_EXPIRE_C15 = 1, QMC_EXPIRE_A4 = 2, QMC_EXPIRE_ADJOINT = 4 };
typedef struct {
    int gj_panel;
    int c15_walkers;
    int a4_mode;
    double a4_kappa_max;
    int c15_mode;
    int bw_walkers;
    double wait_s;
    int expire_walker;
    int expire_kernels;
    double f64_kappa_max;
} qmc_tiles;
int qmc_system_set_tiles(qmc_system *sys, const qmc_tiles *tiles);
int qmc_system_get_tiles(const qmc_system *sys, qmc_tiles *tiles);

/* Copy the per-shell R2 used for screening to host memory [n_shell]. */
int qmc_system_shell_r2(const qmc_system *sys, double *R2_host);

/*
 * qmc_workspace_size -- device scratch needed by qmc_walkers_eval for
 * `n_walk` walkers at `precision` (bytes).  A smaller workspace is allowed:
 * the walkers are then processed in consecutive chunks that fit, down to
 * one walker; below that the call fails with QMC_ERR_CAPACITY.
 */
int qmc_workspace_size(const qmc_system *sys, int n_walk, int precision, size_t *bytes);

/* Outputs of one evaluation, device memory owned by the caller. */
typedef struct {
    double *logpsi;    /* [W]  log|Psi| = log|Det_up| + log|Det_dn| (+ J)  (required) */
    double *sign;      /* [W]  sign of Psi (0 if singular)            (required) */
    double *logabs;    /* [W][2] log|Det_up|, log|Det_dn|             (optional) */
    double *drift;     /* [W][N][3] grad Psi / Psi, Eq. (2)           (required) */
    double *e_loc;     /* [W]  E_L, Eq. (4)                           (required) */
    double *e_parts;   /* [W][4] T, V_en, V_ee, V_nn                  (optional) */
    uint32_t *status;  /* [W]  QMC_STATUS_* bits                      (required) */
    double *dinv;      /* [W][n_up*n_up + n_dn*n_dn] D^-1 per spin, rows = electrons,
                          columns = MOs ((D^-1)_{ek}, D_{ke} = phi_k(r_e)) (optional;
                          qmc_logpsi_backward reads it)                          */
} qmc_eval_out;

/*
 * qmc_walkers_eval -- steps a1..a6 for W walkers.
 *   R         device [W][N][3] FP64 electron positions
 *   precision QMC_PREC_F64 or QMC_PREC_MIXED
 *   ws        device scratch of ws_bytes (see qmc_workspace_size); contents
 *             are overwritten; it must not be in use by another call
 * Errors: QMC_ERR_INVALID (W < 0, NULL required output, unknown precision),
 *         QMC_ERR_CAPACITY (workspace below one walker), QMC_ERR_CUDA.
 */
int qmc_walkers_eval(const qmc_system *sys, int n_walk, const double *R, int precision,
                     const qmc_eval_out *out, void *ws, size_t ws_bytes, qmc_stream_t stream);

/*
 * qmc_walkers_eval_timed -- qmc_walkers_eval that also measures its stages
 * with CUDA events recorded on `stream` between the kernel launches:
 *   stage_ms[0] a1-a3 (screening, AO evaluation, products)
 *   stage_ms[1] a4 (log|det|, sign, inverse)
 *   stage_ms[2] a5-a6 (drift, energies)
 *   stage_ms[3] their sum
 *   stage_ms[4] mixed path: shell masks (a1)
 *   stage_ms[5] mixed path: C1 and C5 products; FP64 path: all of a1-a3
 *   stage_ms[6] mixed path: tensor-core C2..C4 products
 *   stage_ms[7] 0 (reserved)
 * (host float[8], summed over walker chunks).  Blocks until the work has
 * finished.  Same arguments and errors as qmc_walkers_eval.
 */
int qmc_walkers_eval_timed(const qmc_system *sys, int n_walk, const double *R, int precision,
                           const qmc_eval_out *out, void *ws, size_t ws_bytes, qmc_stream_t stream,
                           float *stage_ms);

/*
 * qmc_walkers_eval_static -- qmc_walkers_eval for callers that cannot
 * allocate device memory (for example code running under a memory manager
 * that owns the whole device, a latency-critical loop that must not hit
 * cudaMalloc's implicit synchronisation, or a plug-in whose host forbids
 * driver allocations).  The paper has no counterpart; it is a deployment
 * convenience.  It allocates nothing: its scratch is one fixed device array
 * of QMC_STATIC_SCRATCH_BYTES (64 MiB) inside the library, which every device
 * that loads the library holds until the process exits.
 *   - Walkers are processed in chunks that fit the array; a system whose
 *     single walker needs more scratch than that (e.g. 1731 electrons in
 *     QMC_PREC_F64) is rejected with QMC_ERR_CAPACITY and a message giving
 *     the size.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress), and so does the first call after that device's
 *     CUDA context was destroyed and created again; make that first call
 *     before any stream capture.
 *   - n_walk == 0 returns QMC_OK at once (after checking sys and out), as
 *     qmc_walkers_eval does.
 *   - All calls share the one array and it keeps the last call's contents:
 *     calls that overlap on the GPU (other streams, other threads) race and
 *     corrupt each other's results; serialise them.
 * Arguments, outputs and other errors as for qmc_walkers_eval.
 */
#define QMC_STATIC_SCRATCH_BYTES (64u * 1024u * 1024u)
int qmc_walkers_eval_static(const qmc_system *sys, int n_walk, const double *R, int precision,
                            const qmc_eval_out *out, qmc_stream_t stream);

/*
 * Several systems in one step (mixed batch): each segment is one system's
 * walkers with its own device positions and outputs.  Walkers of different
 * systems are independent (Sec. II.B), so the segments run concurrently on
 * internal streams forked from and joined back into `stream`.
 */
typedef struct {
    const qmc_system *sys;
    int n_walk;
    const double *R;       /* device [n_walk][N][3] */
    qmc_eval_out out;      /* device outputs, as for qmc_walkers_eval */
} qmc_segment;

/* Scratch for qmc_batch_eval: the sum of every segment's full workspace. */
int qmc_batch_workspace_size(const qmc_segment *segs, int n_seg, int precision, size_t *bytes);

/* a1..a6 for every segment (all systems on one device); ws of
 * qmc_batch_workspace_size bytes (QMC_ERR_CAPACITY if smaller). */
int qmc_batch_eval(const qmc_segment *segs, int n_seg, int precision, void *ws, size_t ws_bytes,
                   qmc_stream_t stream);

/* qmc_batch_eval captured once into a CUDA graph; each qmc_graph_launch
 * replays the whole mixed batch (same pointers: refill the R buffers in
 * place between launches).  Creation synchronises the device. */
typedef struct qmc_graph qmc_graph;
int qmc_batch_graph_create(const qmc_segment *segs, int n_seg, int precision, void *ws, size_t ws_bytes,
                           qmc_graph **out);
int qmc_graph_launch(qmc_graph *g, qmc_stream_t stream);
int qmc_graph_free(qmc_graph *g);

/*
 * qmc_logpsi_backward -- a7, the adjoint of log|Psi| with respect to the MO
 * coefficients, weighted over walkers:
 *   dA_s[mu][k] = sum_w g_w sum_{e in spin s} (D^-1)_{w,ek} chi_mu(r_{w,e})
 * (from d log|det D| / dD_{ke} = (D^-1)_{ek} and D_{ke} = sum_mu a_{k mu} chi_mu(r_e)).
 * chi is recomputed from R (screened exactly as in the forward pass), D^-1 is
 * the forward pass's `dinv` output.  g = 1/W gives d<log|Psi|>/dA;
 * g_w = 2 (E_L,w - <E_L>)/W gives the E_L-weighted gradient.
 *   R     device [W][N][3] f64;  dinv  device [W][n_up^2 + n_dn^2] f64
 *   g     device [W] f64;  walkers whose status is non-zero must have g_w = 0
 *   dA_up device [n_ao][n_up], dA_dn [n_ao][n_dn], FP64 (overwritten)
 */
int qmc_logpsi_backward(const qmc_system *sys, int n_walk, const double *R, const double *dinv,
                        const double *g, double *dA_up, double *dA_dn, qmc_stream_t stream);

/*
 * qmc_backward_workspace_size -- device scratch (bytes) that
 * qmc_logpsi_backward_ex needs to process `n_walk` walkers in one pass at
 * `precision` (0 for QMC_PREC_F64; passes hold at most 512 walkers).
 */
int qmc_backward_workspace_size(const qmc_system *sys, int n_walk, int precision, size_t *bytes);

/*
 * qmc_logpsi_backward_ex -- a7 with a choice of arithmetic.
 *   QMC_PREC_F64    exactly qmc_logpsi_backward (ws unused).
 *   QMC_PREC_MIXED  the same sum as a contraction over the (walker, electron)
 *                   pairs inside the screening radius of an AO block, on the
 *                   tcgen05 tensor cores: D^-1 rounded to FP32 and g_w chi_mu
 *                   evaluated in FP32, both split exactly into three BF16
 *                   slices, the six slice products of order <= 2 accumulated
 *                   in FP32 per block of qmc_tiles.bw_walkers walkers (8 by
 *                   default), the blocks summed in FP64.
 *                   Each term carries a relative error of a few 2^-24.
 * Arguments as qmc_logpsi_backward, plus
 *   ws, ws_bytes  device scratch (qmc_backward_workspace_size); a smaller
 *                 workspace processes the walkers in several passes, down to
 *                 one walker (below that: QMC_ERR_CAPACITY).
 * Layouts and ownership as qmc_logpsi_backward; asynchronous on `stream`.  A
 * bounded device wait that expires (2 s) leaves NaN in the rows of dA that
 * the waiting CTA owned.
 * Errors: QMC_ERR_INVALID (unknown precision, NULL pointer), QMC_ERR_CAPACITY,
 *         QMC_ERR_CUDA.
 */
int qmc_logpsi_backward_ex(const qmc_system *sys, int n_walk, const double *R, const double *dinv,
                           const double *g, int precision, double *dA_up, double *dA_dn, void *ws,
                           size_t ws_bytes, qmc_stream_t stream);

/*
 * qmc_screen_ao -- steps a1+a2 alone, for inspection and parity tests.
 * For each walker w and electron e: cnt[w][e] = number of non-zero AOs,
 * idx[w][e][0..cnt) their indices in ascending order, B[w][e][l][k] the
 * value (l=0), gradient (l=1..3) and Laplacian (l=4) of AO idx[w][e][k], FP64.
 * Entries k >= min(cnt, cap) are left untouched; cnt may exceed cap.
 *   R device [W][N][3];  cnt device [W][N] i32;  idx device [W][N][cap] i32;
 *   B device [W][N][5][cap] f64 (may be NULL)
 */
int qmc_screen_ao(const qmc_system *sys, int n_walk, const double *R, int cap, int32_t *cnt,
                  int32_t *idx, double *B, qmc_stream_t stream);

/*
 * qmc_shell_masks -- step a1 of the mixed path alone: bit (sh & 31) of word
 * (sh >> 5) of masks[w][e] is set iff shell sh is active for electron e of
 * walker w (Sec. III: d^2 < R^2_shell and d^2 < R^2_atom, the same
 * correctly rounded FP64 decisions as qmc_screen_ao).  *mask_words receives
 * the number of 32-bit words per electron, ceil(n_shell / 32); with
 * masks == NULL only that number is returned.
 *   R device [W][N][3] f64;  masks device [W][N][mask_words] u32
 */
int qmc_shell_masks(const qmc_system *sys, int n_walk, const double *R, uint32_t *masks, int *mask_words,
                    qmc_stream_t stream);

/*
 * qmc_slater_matrices -- steps a1..a3 alone: C_l[e][k] = d_l phi_k(r_e),
 * l = 0 value, 1..3 gradient, 4 Laplacian; per walker the up block
 * [5][n_up][n_up] followed by the down block [5][n_dn][n_dn], FP64, at the
 * given precision (the mixed path's values are widened from its own result).
 *   C device [W][5*(n_up^2 + n_dn^2)] f64;  ws/ws_bytes as for qmc_walkers_eval.
 */
int qmc_slater_matrices(const qmc_system *sys, int n_walk, const double *R, int precision,
                        double *C, void *ws, size_t ws_bytes, qmc_stream_t stream);

/*
 * qmc_det_inverse -- step a4 alone on a batch of `batch` FP64 n x n matrices
 * X (row-major, X[e][k] = phi_k(r_e), i.e. the transpose of the paper's
 * D_{ke}): log|det X|, sign, and Dinv = X^-T (= D^-1, rows = electrons).
 * Gauss-Jordan elimination with partial pivoting in panels of 16 columns;
 * the pivots are those of LU with partial pivoting.  X is overwritten.
 *   X, Dinv device [batch][n][n];  logabs, sign device [batch];  singular
 *   device [batch] u32 (1 if an exact zero pivot occurred; Dinv is then NaN)
 *   1 <= n <= 1024.
 */
int qmc_det_inverse(int batch, int n, double *X, double *Dinv, double *logabs, double *sign,
                    uint32_t *singular, qmc_stream_t stream);

/*
 * qmc_multidet_eval -- a1..a6 for a multi-determinant trial function (Sec. II.C,
 * Eq. psit): Psi = e^J sum_K c_K Det_K,up Det_K,dn, K = 0..n_det-1 (1..64).
 * Determinant K is a loaded system with the MO coefficients of its
 * configuration (e.g. an excitation of the reference); all share the device,
 * the electron counts, nuclei, basis and Jastrow factor (QMC_ERR_INVALID
 * otherwise).  Each determinant is evaluated with qmc_walkers_eval's kernels,
 * then combined per walker: with L_K = log|Psi_K|, s_K its sign, L = max L_K
 * over the determinants that are not singular, S = sum_K c_K s_K e^{L_K - L}
 * and w_K = c_K s_K e^{L_K - L} / S:
 *   log|Psi| = L + log|S|, sign = sign(S), drift = sum_K w_K b_K,
 *   T = sum_K w_K T_K, E_L = sum_K w_K E_L,K (the potential is the same).
 * S == 0 (a node of the expansion) or every determinant singular: status
 * SINGULAR_UP | SINGULAR_DN, log|Psi| = -inf.  out->logabs (optional) is NaN
 * (no per-spin determinant exists); out->dinv must be NULL.
 *   coef host [n_det]; R device [W][N][3]; ws of qmc_multidet_workspace_size
 *   bytes (per-determinant results and one evaluation's workspace; a smaller
 *   evaluation part processes the walkers in chunks).  Cost: n_det evaluations
 *   (an excitation-based update of D^-1 per determinant is not used).
 */
int qmc_multidet_workspace_size(const qmc_system *const *dets, int n_det, int n_walk, int precision,
                                size_t *bytes);
int qmc_multidet_eval(const qmc_system *const *dets, const double *coef, int n_det, int n_walk, const double *R,
                      int precision, const qmc_eval_out *out, void *ws, size_t ws_bytes, qmc_stream_t stream);

/*
 * ---------------------------------------------------------------------------
 * The Monte Carlo step around the evaluation (Sec. II.A and II.B): fixed-node
 * diffusion Monte Carlo with a constant number of walkers.
 *
 * Random numbers come from Philox4x64-10 (Salmon, Moraes, Dror and Shaw,
 * SC'11), a counter-based generator, so a walker's numbers depend only on
 * (seed, step, walker, component), never on the launch:
 *   move  key (seed, 0), counter (j, walker, step, 0): block j gives the
 *         normals of components 4j..4j+3 of the walker's 3N (component 3e + c
 *         is coordinate c of electron e) through two Box-Muller pairs,
 *         u1 = ((x0 >> 11) + 1) 2^-53, u2 = (x1 >> 11) 2^-53,
 *         (sqrt(-2 ln u1) cos 2 pi u2, sqrt(-2 ln u1) sin 2 pi u2), then (x2, x3);
 *   draws key (seed, 1), counter (j >> 2, step, 0, 0): output j & 3 is the
 *         64-bit uniform integer of draw j of the reconfiguration.
 * ---------------------------------------------------------------------------
 */

/* The state of W walkers, device memory: positions and what the evaluation
 * returned for them. */
typedef struct {
    double *R;         /* [W][N][3] */
    double *drift;     /* [W][N][3] grad Psi / Psi, Eq. (2) */
    double *e_loc;     /* [W] E_L, Eq. (4) */
    double *logpsi;    /* [W] */
    double *sign;      /* [W] */
    uint32_t *status;  /* [W] QMC_STATUS_* bits */
} qmc_walker_state;

/*
 * qmc_dmc_move -- Eq. (1): R_new = R + tau b(R) + sqrt(tau) eta for W walkers
 * of N electrons, eta the Philox/Box-Muller normals of the "move" stream.
 * Each component is rounded as written, (R + tau b) + sqrt(tau) eta, without
 * fused multiply-adds.  R, drift, R_new device [W][N][3] f64 (R_new may not
 * alias R).  step_ptr: NULL, or a device uint64 read in place of `step` (so a
 * captured CUDA graph can advance it, see qmc_dmc_step).
 */
int qmc_dmc_move(int n_walk, int n_elec, const double *R, const double *drift, double tau, uint64_t seed,
                 uint64_t step, const uint64_t *step_ptr, double *R_new, qmc_stream_t stream);

/*
 * qmc_dmc_weight -- Eq. (3) with the fixed-node rule (Sec. II.A: the nodes
 * of Psi_T are infinitely repulsive barriers).  accept[w] = 1 iff the old
 * walker is valid (status 0, sign != 0), the proposed one is valid and Psi_T
 * kept its sign; weight[w] = exp(-(((E' - E_T) + (E_old - E_T)) * (tau / 2)))
 * with E' = e_new[w] if accepted, else e_old[w]; an invalid old walker gets
 * weight 0.  All arrays device [W]; e_trial_ptr: NULL or a device double read
 * in place of e_trial.
 */
int qmc_dmc_weight(int n_walk, const double *e_old, const double *sign_old, const uint32_t *status_old,
                   const double *e_new, const double *sign_new, const uint32_t *status_new, double tau,
                   double e_trial, const double *e_trial_ptr, double *weight, uint32_t *accept,
                   qmc_stream_t stream);

/*
 * qmc_srmc_reconfigure -- Sec. II.B: draw M = W walkers among the W with
 * probabilities p_k = w_k / sum_i w_i, in exact integer arithmetic:
 * q_k = floor(2^40 w_k / max_i w_i) (a weight that is not finite or not
 * positive counts 0), C_k = q_0 + ... + q_k (64-bit, exact), draw j takes the
 * first k with C_k > floor(U_j C_{W-1} / 2^64), U_j the 64-bit integer of the
 * "draws" stream.  The indices are thus a function of the weights, seed and
 * step alone.  If every weight is 0 the population is kept (idx[j] = j).
 *   weight device [W] f64; idx device [W] i32 (new walker j copies old walker
 *   idx[j]); stats NULL or device [4] f64: sum of the counted weights, their
 *   number, 0, 0; ws device scratch of at least 8 W bytes.
 * One CTA: W up to 2^24.
 */
int qmc_srmc_reconfigure(int n_walk, const double *weight, uint64_t seed, uint64_t step, const uint64_t *step_ptr,
                         int32_t *idx, double *stats, void *ws, size_t ws_bytes, qmc_stream_t stream);

/* Parameters of one DMC step.  step_ptr / e_trial_ptr (device, optional)
 * replace step / e_trial when not NULL; qmc_dmc_step then adds 1 to *step_ptr
 * in its last kernel, so a CUDA graph captured from one step replays the
 * following ones. */
typedef struct {
    double tau;
    double e_trial;
    uint64_t seed;
    uint64_t step;
    int precision;              /* of the evaluation: QMC_PREC_* */
    uint64_t *step_ptr;
    const double *e_trial_ptr;
} qmc_dmc_params;

/* Device scratch (bytes) of qmc_dmc_step for W walkers: the evaluation's
 * workspace (qmc_workspace_size) plus the proposed walkers, weights, accept
 * flags, draws and the reconfiguration's sums. */
int qmc_dmc_workspace_size(const qmc_system *sys, int n_walk, int precision, size_t *bytes);

/*
 * qmc_dmc_step -- one fixed-node DMC step with constant population, in the
 * paper's order: move every walker (Eq. 1), evaluate the proposed positions
 * (a1..a6: drift Eq. 2, E_L Eq. 4), keep or reject each move and weigh it
 * (Eq. 3, qmc_dmc_weight), draw the new population (Sec. II.B,
 * qmc_srmc_reconfigure), and copy the drawn walkers' state to `out`.
 *   in   the current walkers (as evaluated: drift, e_loc, logpsi, sign, status
 *        of their positions); out: the next generation, same layout, must not
 *        alias `in`.
 *   stats NULL or device [4] f64: sum_k w_k, the number of walkers with a
 *        positive weight, sum_k w_k E_L,k (E_L of the kept state, before the
 *        draw: the numerator of the generation's weighted average), the number
 *        of accepted moves.  The paper's global weight of a generation is
 *        stats[0] / W; its product over the preceding generations weighs the
 *        averages (left to the caller).
 * Asynchronous on `stream`; nothing is allocated; capturable in a CUDA graph
 * with step_ptr set (the first call of a system should come before the
 * capture, as for qmc_walkers_eval).
 * Errors: QMC_ERR_INVALID (bad arguments, tau <= 0), QMC_ERR_CAPACITY
 * (workspace below qmc_dmc_workspace_size), QMC_ERR_CUDA.
 */
int qmc_dmc_step(const qmc_system *sys, int n_walk, const qmc_walker_state *in, const qmc_walker_state *out,
                 const qmc_dmc_params *params, double *stats, void *ws, size_t ws_bytes, qmc_stream_t stream);

/* Message of the last failed call on the calling thread ("" if none). */
const char *qmc_last_error(void);

/* Library version string. */
const char *qmc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* QMCGB_H */
