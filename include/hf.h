/*
 * hf.h - C-ABI of the GB300 (sm_103a) direct-SCF Fock-build library.
 *
 * The library builds the closed-shell Hartree-Fock Fock matrix
 *     F = H + J - K/2,  J_mn = sum_ls P_ls (mn|ls),  K_mn = sum_ls P_ls (ml|ns)
 * (Section 3 of Mironov et al., SC17, "An efficient MPI/OpenMP
 * parallelization of the Hartree-Fock method for the second generation of
 * Intel Xeon Phi processor": Eq. FC = eSC and the two-electron part of F) by
 * the direct-SCF algorithm of Section 4: the symmetry-unique shell quartets of
 * Algorithm 1, Cauchy-Schwarz screened, each electron-repulsion integral
 * applied to the six Fock elements of Eq. 1a-1f.  Integrals are evaluated on
 * the GPU by Obara-Saika / Head-Gordon-Pople recurrences over contracted
 * Cartesian Gaussians (the paper treats eri() as a black box).
 *
 * Conventions (every entry point):
 *   - Units are atomic units (bohr, hartree).
 *   - Matrices are N x N, row-major, FP64, N = number of Cartesian basis
 *     functions.  Basis functions are ordered by shell, and inside a shell by
 *     Cartesian component: p = x, y, z; d = xx, xy, xz, yy, yz, zz.
 *   - Each contracted Cartesian component is normalised so that S_mm = 1;
 *     contraction coefficients multiply normalised primitives.
 *   - P is the total (closed-shell) density, P = 2 C_occ C_occ^T.
 *   - Matrix arguments are host pointers unless HF_PTR_DEVICE is set in
 *     flags, in which case they are device pointers on the context's device.
 *     The caller owns every buffer it passes; the library never keeps a
 *     pointer to a caller buffer after a call returns.
 *   - Every call returns HF_OK (0) or a negative status and never aborts.
 *     Outputs are written only on success.  hf_last_error() describes the
 *     most recent failure on the calling thread.
 *   - All device work is ordered on the stream given to hf_create; calls
 *     return after that stream has finished the call's work.
 */
#ifndef HF_H
#define HF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define HF_OK 0
#define HF_E_INVALID -1     /* bad argument: null pointer, NaN/Inf, asymmetric P, bad sizes */
#define HF_E_UNSUPPORTED -2 /* l > 2, too many primitives, no sm_103a device */
#define HF_E_NOMEM -3       /* device or host allocation failed */
#define HF_E_CUDA -4        /* a CUDA runtime call failed */
#define HF_E_TIMEOUT -5     /* a bounded device wait gave up */
#define HF_E_NOCONV -6      /* SCF did not converge within max_iter */

/* ----------------------------------------------------------------- flags */
#define HF_PTR_HOST 0   /* matrix arguments are host pointers */
#define HF_PTR_DEVICE 1 /* matrix arguments are device pointers */
#define HF_TIMING 2     /* fill the per-kernel device times of hf_stats */
#define HF_FP64_ONLY 8  /* hf_fock_build: evaluate the FP32 part of a mixed system in FP64 too */
#define HF_DENSITY_SCREEN 16 /* hf_fock_build_partial: also skip quartets whose Schwarz bound times the
                                largest |P| of the six density blocks they touch (x4) is below schwarz_tau */
#define HF_RYS 32            /* hf_fock_build, hf_fock_build_partial: evaluate the FP64 quartets of all five
                                classes of total angular momentum L >= 6 ((dp|dp), (dd|pp), (dd|ds), (dd|dp),
                                (dd|dd)) by Rys quadrature (L/2 + 1 nodes of the Boys weight) instead of the
                                Obara-Saika vertical recurrence; the contraction, horizontal recurrence and
                                digestion are shared, so results agree to rounding.  Without HF_RYS or
                                HF_OBARA_SAIKA the builds use Rys for the four of them where it is faster
                                ((dp|dp), (dd|ds), (dd|dp), (dd|dd)) and Obara-Saika for (dd|pp).  FP32
                                launches and the batched builds always use Obara-Saika. */
#define HF_OBARA_SAIKA 64    /* hf_fock_build, hf_fock_build_partial: Obara-Saika for every class (no Rys);
                                with HF_RYS as well, HF_OBARA_SAIKA wins */

typedef struct hf_ctx hf_ctx;       /* one device + one stream + constant tables */
typedef struct hf_system hf_system; /* one molecule: basis, pairs, screening plan, 1e matrices */

/* Nuclei.  Z[n_atoms] charges; xyz[3*n_atoms] positions in bohr.  Host memory. */
typedef struct {
    int32_t n_atoms;
    const int32_t* Z;
    const double* xyz;
} hf_geometry;

/* Contracted Cartesian shells (Section 4.1's "shell": functions on one atom
 * sharing exponents).  atom[s] atom index, l[s] in 0..2 or HF_SP_SHELL,
 * nprim[s] in 1..8, exps/coefs: sum(nprim) primitive exponents and
 * coefficients, shell after shell.  An sp (L) shell, as in split-valence
 * bases such as 6-31G(d) (the paper's basis, Section 5), is an s and a p
 * shell sharing exponents: coefs holds its s coefficients and coefs_p its p
 * coefficients (coefs_p is read only at sp shells and may be NULL when there
 * are none); its functions are ordered s, x, y, z.  Host memory. */
#define HF_SP_SHELL -1
typedef struct {
    int32_t n_shells;
    const int32_t* atom;
    const int32_t* l;
    const int32_t* nprim;
    const double* exps;
    const double* coefs;
    const double* coefs_p;
} hf_basis;

/* Screening and precision thresholds.
 *   schwarz_tau : skip a shell quartet when Q_ij * Q_kl < schwarz_tau
 *                 (Algorithm 1's schwartz(i,j,k,l)); 0 disables screening.
 *   fp32_cutoff : evaluate a quartet's integrals in FP32 when
 *                 Q_ij * Q_kl < fp32_cutoff (accumulation stays FP64);
 *                 0 keeps every quartet in FP64.
 *   prim_tau    : skip a primitive quartet when B_ab * B_cd < prim_tau, with
 *                 B = sqrt(max |[ab|ab]|) the Schwarz bound of one primitive
 *                 pair (normalised components); 0 evaluates every primitive
 *                 quartet.  Each skipped primitive quartet changes any
 *                 integral by at most prim_tau. */
typedef struct {
    double schwarz_tau;
    double fp32_cutoff;
    double prim_tau;
} hf_thresholds;

#define HF_NUM_CLASSES 21

/* Work and time accounting of one Fock build.  Class c is the c-th (X|Y)
 * pair of pair classes ss, ps, pp, ds, dp, dd with X >= Y, in the order
 * (ss|ss), (ps|ss), (ps|ps), (pp|ss), (pp|ps), (pp|pp), (ds|ss), ... */
typedef struct {
    int64_t quartets_unscreened; /* symmetry-unique shell quartets before screening */
    int64_t quartets_fp64;       /* shell quartets evaluated in FP64 */
    int64_t quartets_fp32;       /* shell quartets evaluated in FP32 */
    int64_t class_quartets_fp64[HF_NUM_CLASSES];
    int64_t class_quartets_fp32[HF_NUM_CLASSES];
    double flops_fp64; /* algorithmic FP64 operations of the ERI kernels */
    double flops_fp32; /* algorithmic FP32 operations of the ERI kernels */
    float ms_class_fp64[HF_NUM_CLASSES]; /* device time per class kernel (HF_TIMING) */
    float ms_class_fp32[HF_NUM_CLASSES];
    float ms_eri;   /* device time of all ERI kernels (HF_TIMING) */
    float ms_total; /* device time of the whole build (HF_TIMING) */
    double class_flops_fp64[HF_NUM_CLASSES]; /* algorithmic operations per class kernel */
    double class_flops_fp32[HF_NUM_CLASSES];
    int32_t kernels_launched; /* library kernels launched by this call */
    int64_t prim_quartets_fp64; /* primitive quartets evaluated (after primitive screening) */
    int64_t prim_quartets_fp32;
} hf_stats;

/* Sizes of a system. */
typedef struct {
    int32_t n_atoms, n_shells, n_bf, n_electrons;
    int64_t n_pairs;             /* unordered shell pairs */
    int64_t n_significant_pairs; /* pairs with Q_ij * max Q >= schwarz_tau */
    int64_t quartets_unscreened;
    int64_t quartets_fp64, quartets_fp32; /* after screening */
    double E_nn;                          /* nuclear repulsion energy */
    double Q_max;
    int64_t device_bytes; /* device memory held by the system */
} hf_system_info;

/* ------------------------------------------------------------ lifecycle */

/* Create a context on CUDA device `device` that orders all work on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).  The
 * stream is borrowed and must outlive the context.  Builds the Boys-function
 * tables on the device and looks up the address of the fixed scratch of
 * hf_fock_build_noalloc, which makes the driver reserve that array (about
 * 7.3 MB per device, held until the process exits) here rather than in a
 * later call.  Errors: HF_E_INVALID (ctx NULL),
 * HF_E_UNSUPPORTED (device is not compute capability 10.3), HF_E_CUDA. */
int hf_create(hf_ctx** ctx, int device, void* cuda_stream);

/* Release a context (NULL is ignored).  If systems created on it are still
 * alive, the context stays usable by them and is released together with the
 * last of them. */
void hf_destroy(hf_ctx* ctx);

/* Short text for a status code; never NULL. */
const char* hf_strerror(int status);

/* Message of the last failure on the calling thread ("" if none). */
const char* hf_last_error(void);

/* ---------------------------------------------------------------- system */

/* Set up one molecule (Section 3: one-electron part, O(N^2), done once per
 * geometry): normalisation, S, H = T + V, E_nn, all shell pairs with their
 * primitive-pair data and Schwarz bounds, the significant-pair lists sorted
 * by angular class and bound, and the per-class quartet schedule for the
 * given thresholds.  Geometry and basis are read from host memory and not
 * kept.  Errors: HF_E_INVALID (null/negative sizes, atom index out of
 * range, non-positive exponent, NaN, negative threshold, sp shell without
 * coefs_p), HF_E_UNSUPPORTED (l > 2, nprim > 8), HF_E_NOMEM, HF_E_CUDA.
 * The system holds an sp shell as an s shell followed by a p shell with the
 * same exponents, so hf_system_info counts both. */
int hf_system_create(hf_ctx* ctx, const hf_geometry* geom, const hf_basis* basis, const hf_thresholds* th,
                     hf_system** sys);

/* Release a system (NULL is ignored). */
void hf_system_destroy(hf_system* sys);

/* Sizes and counts of a system. */
int hf_system_get_info(const hf_system* sys, hf_system_info* info);

/* Overlap S and core Hamiltonian H = T + V (N x N).  Either output may be
 * NULL.  flags: HF_PTR_DEVICE for device outputs. */
int hf_one_electron(hf_system* sys, double* S, double* H, int flags);

/* ------------------------------------------------------------ Fock build */

/* One direct-SCF Fock build (Algorithms 1-3, Eq. 1a-1f).
 *   P      [N*N] total density, symmetric to 1e-12 relative, finite.
 *   F      [N*N] output H + J - K/2 (may be NULL).
 *   J, K   [N*N] outputs (may be NULL).
 *   E_elec host scalar output 1/2 sum P (H + F) (may be NULL).
 *   stats  host output (may be NULL); HF_TIMING adds device times.
 * flags: HF_PTR_DEVICE (P, F, J, K are device pointers), HF_TIMING,
 * HF_FP64_ONLY, HF_RYS, HF_OBARA_SAIKA.  The density check runs on the device:
 * the host waits once, after the whole build, and a rejected density leaves
 * every output untouched.
 * Errors: HF_E_INVALID (NULL sys/P, P not finite or not symmetric),
 * HF_E_NOMEM, HF_E_CUDA. */
int hf_fock_build(hf_system* sys, const double* P, double* F, double* J, double* K, double* E_elec, hf_stats* stats,
                  int flags);

/* Device microbenchmarks that give the roofline denominators of the build:
 * FP64 and FP32 FMA throughput (independent FMA chains on every SM; the ERI
 * kernels of Section 3's integral step are bound by the FP64 pipe) and FP64
 * atomic-add throughput into an 8 MB array (the digestion of Eq. 1a-1f),
 * random and coalesced addresses.  Each figure is the best of three timed
 * launches after a warm-up, on the context's stream, with CUDA events; it
 * takes well under a second.  Rates are per second over the whole GPU.
 * Errors: HF_E_INVALID (NULL argument), HF_E_NOMEM, HF_E_CUDA. */
typedef struct {
    double fp64_fma_gflops;
    double fp32_fma_gflops;
    double red_add_f64_random_gops;
    double red_add_f64_coalesced_gops;
    double sm_max_mhz;
    int32_t num_sms;
    int32_t pad;
} hf_peaks;
int hf_measure_peaks(hf_ctx* ctx, hf_peaks* out);

/* Accumulators of the ERI digestion (the paper's shared vs private Fock
 * matrices, Section 3 and Table 3, mapped to GPU thread blocks).
 *   copies == 1 (default): every thread block adds its quartets' Eq. 1a-1f
 *     updates into one shared pair of N x N accumulators with FP64 atomics;
 *   copies  > 1: block b adds into private copy b % copies; the copies are
 *     summed after the ERI launches.  Costs 2 * copies * N * N * 8 bytes of
 *     device memory plus zeroing and summing them on every build.
 * Applies to hf_fock_build, hf_fock_build_partial and hf_scf_run (not to the
 * batched or allocation-free builds).  Results equal those with one copy up
 * to the order of FP64 additions.
 * Errors: HF_E_INVALID (NULL system, copies outside 1..4096), HF_E_NOMEM (the
 * copies do not fit; the system is left with one shared copy). */
int hf_system_set_fock_copies(hf_system* sys, int32_t copies);

/* One shard of the Fock build for multi-device or multi-process use: the
 * quartets [n s / S, n (s+1) / S) of every angular-class launch (n = that
 * launch's screened quartet count), giving partial J and K.  The sum over
 * s = 0..S-1 of the partial J (K) is the full J (K), so F = H + sum_s J_s -
 * 1/2 sum_s K_s: the counterpart of the paper's per-rank partial Fock matrix
 * and ddi_gsumf (Algorithms 1-3), with the sum left to the caller (for
 * example one allreduce of J and K).  J, K: [N*N] outputs (required).
 * flags: HF_PTR_DEVICE, HF_FP64_ONLY, HF_RYS, HF_OBARA_SAIKA, HF_DENSITY_SCREEN (density-weighted
 * Schwarz screening: the J and K of a density difference, as in incremental
 * SCF builds).  Errors: HF_E_INVALID (bad shard, NULL pointer, P not finite
 * or not symmetric), HF_E_CUDA. */
int hf_fock_build_partial(hf_system* sys, const double* P, int shard, int n_shards, double* J, double* K, int flags);

/* Assembly of a sharded build (the step after the paper's ddi_gsumf in
 * Algorithms 2/3): F = H + J - K/2 from J and K already summed over every
 * shard of hf_fock_build_partial (for example by one allreduce of J and one
 * of K), and E_elec = 1/2 sum P (H + F) when E_elec is not NULL.
 *   P      [N*N] total density (required only with E_elec).
 *   J, K   [N*N] summed Coulomb and exchange matrices.
 *   F      [N*N] output.
 *   E_elec host scalar output or NULL.
 * flags: HF_PTR_DEVICE (P, J, K, F are device pointers).  Errors:
 * HF_E_INVALID (NULL argument, E_elec without P, J or K not finite), HF_E_CUDA. */
int hf_fock_assemble(hf_system* sys, const double* P, const double* J, const double* K, double* F, double* E_elec,
                     int flags);

/* ------------------------------------------------------------------- SCF */

/* Options of hf_scf_run (zero-initialise, then set what differs):
 *   n_occ      doubly occupied orbitals (0: n_electrons / 2)
 *   max_iter   Fock builds at most (0: 100)
 *   e_tol      |E_k - E_{k-1}| threshold in Eh (0: 1e-9)
 *   d_tol      RMS(P_k - P_{k-1}) threshold (0: 1e-6)
 *   diis_size  Pulay DIIS history length, 0..16 (0 with diis_off = 1 disables)
 *   diis_off   1 disables DIIS
 *   mixed_switch  for a system with fp32_cutoff > 0: Fock builds use the
 *              mixed FP32/FP64 split until |dE| < mixed_switch (0: 1e-5),
 *              then every later build is FP64 only (HF_FP64_ONLY) and the
 *              DIIS history restarts; convergence is only declared on FP64
 *              builds, so the final energy is that of the plain FP64 method.
 *   incremental  1: between full rebuilds, J and K are updated with the J and
 *              K of P_k - P_ref (hf_fock_build_partial with HF_DENSITY_SCREEN),
 *              so small density changes skip most quartets.  Once |dE| falls
 *              below incremental_switch (or the convergence test passes on such
 *              a build), every further build is a full one, the DIIS history
 *              restarts, and convergence is only declared on a full build (so
 *              the final energy is that of the plain method).
 *   rebuild_every  full rebuild period of the incremental mode (0: 8).
 *   incremental_switch  |dE| below which incremental builds stop (0: 1e-5). */
typedef struct {
    int32_t n_occ;
    int32_t max_iter;
    double e_tol;
    double d_tol;
    int32_t diis_size;
    int32_t diis_off;
    double mixed_switch;
    int32_t incremental;
    int32_t rebuild_every;
    double incremental_switch;
} hf_scf_opts;

/* Result of hf_scf_run. */
typedef struct {
    double energy;          /* total energy E_elec + E_nn at the last density (Eh) */
    double E_nn;            /* nuclear repulsion */
    int32_t iterations;     /* Fock builds performed */
    int32_t converged;      /* 1 if both thresholds were met */
    double last_dE, last_dP;
    double seconds_total;   /* host wall time of the call */
    double seconds_fock;    /* of which Fock builds */
    double seconds_diag;    /* of which orthogonalisation + diagonalisation + density */
    int32_t jacobi_sweeps;  /* total Jacobi sweeps of all diagonalisations */
    int32_t n_kept;         /* orthogonal basis size (N unless near-linear dependence) */
    double s_min;           /* smallest overlap eigenvalue */
    int32_t mixed_iterations; /* builds done with the FP32/FP64 split */
    int32_t full_builds;      /* builds from the full density (the rest were incremental) */
} hf_scf_result;

/* Closed-shell SCF (Section 3, Eq. FC = eSC): X = S^-1/2 (canonical
 * orthogonalisation when an overlap eigenvalue is below 1e-8), guess = core
 * Hamiltonian unless P_guess is given, then F(P) by hf_fock_build, Pulay DIIS
 * on FPS - SPF, eigenpairs of X^T F X by the device Jacobi solver,
 * P = 2 C_occ C_occ^T, until |dE| < e_tol and RMS dP < d_tol.
 *   P_guess   [N*N] initial density or NULL
 *   P_out     [N*N] final density (the one F was built from) or NULL
 *   eps_out   [n_kept] orbital energies of the last diagonalisation or NULL
 *   energies  host array of max_iter energies per iteration, or NULL
 *   res       host output (required)
 * flags: HF_PTR_DEVICE for P_guess / P_out / eps_out.  Errors: HF_E_INVALID,
 * HF_E_NOMEM, HF_E_CUDA, HF_E_NOCONV (res and P_out then hold the last
 * iterate). */
int hf_scf_run(hf_system* sys, const hf_scf_opts* opts, const double* P_guess, double* P_out, double* eps_out,
               double* energies, hf_scf_result* res, int flags);

/* Eigen-decomposition of a symmetric n x n matrix A on the device (parallel
 * cyclic Jacobi, the diagonalisation step of Section 3's SCF).  w[n]
 * eigenvalues ascending; V[n*n] row-major with eigenvector j in column j.
 * flags: HF_PTR_DEVICE for device pointers.  Errors: HF_E_INVALID,
 * HF_E_NOMEM, HF_E_CUDA, HF_E_NOCONV (60 sweeps). */
int hf_eigh(hf_ctx* ctx, int n, const double* A, double* w, double* V, int flags);

/* --------------------------------------------------------------- batches */

typedef struct hf_batch hf_batch; /* many independent molecules built together */

#define HF_BATCH_SEQUENTIAL 4 /* hf_fock_build_batch: one hf_fock_build per molecule instead of the graph */

/* Sizes and tuning of a batch. */
typedef struct {
    int32_t n_mol;
    int64_t packed_len; /* sum of N_m^2: length of the packed matrix arrays */
    int64_t n_bf_total;
    int64_t quartets; /* screened shell quartets of one batched build */
    int64_t class_quartets[HF_NUM_CLASSES];
    int32_t block[HF_NUM_CLASSES];         /* threads per block of each class kernel */
    int32_t chunk[HF_NUM_CLASSES];         /* quartets per work-queue grab */
    int32_t blocks_per_sm[HF_NUM_CLASSES]; /* persistent grid = SMs x blocks_per_sm */
} hf_batch_info;

/* Set up n_mol independent molecules (geoms[m], bases[m]; thresholds shared,
 * FP64 integrals: fp32_cutoff is ignored) for batched Fock builds.  The
 * per-iteration work of the whole batch (density scaling, one persistent
 * kernel per angular class over every molecule's quartets fed by a device
 * work queue - the GPU counterpart of Algorithm 1's ddi_dlbnext dynamic load
 * balancing - assembly and energies) is captured once in a CUDA graph.
 * Errors as hf_system_create. */
int hf_batch_create(hf_ctx* ctx, int n_mol, const hf_geometry* geoms, const hf_basis* bases,
                    const hf_thresholds* th, hf_batch** batch);
void hf_batch_destroy(hf_batch* batch);
int hf_batch_get_info(const hf_batch* batch, hf_batch_info* info);

/* off[n_mol + 1]: offset of molecule m's N_m x N_m block in the packed arrays. */
int hf_batch_offsets(const hf_batch* batch, int64_t* off);

/* One Fock build of every molecule.  P and F are packed arrays (molecule m's
 * row-major N_m x N_m block at off[m]); host pointers unless HF_PTR_DEVICE.
 * E_elec: host array of n_mol electronic energies or NULL; ms: host output of
 * the device time of the build or NULL.  HF_BATCH_SEQUENTIAL runs one
 * hf_fock_build per molecule instead (the unbatched reference).  Errors:
 * HF_E_INVALID (NULL argument, a density not finite or not symmetric),
 * HF_E_CUDA. */
int hf_fock_build_batch(hf_batch* batch, const double* P, double* F, double* E_elec, float* ms, int flags);

/* Autotuner: for every class kernel, time each candidate (block size 64/128/
 * 256, chunk 32/128/512 quartets, 2/4/8 blocks per SM) on the class's first
 * quartets - as many as take about 2e10 algorithmic operations, at most
 * sample_quartets (0: 2e6) - and keep the fastest; choices are read
 * from and written to cache_path (one "class block chunk blocks_per_sm" line
 * per class) when it is not NULL.  Re-captures the graph.  Errors: HF_E_INVALID,
 * HF_E_CUDA. */
int hf_batch_tune(hf_batch* batch, const char* cache_path, int64_t sample_quartets);

/* --------------------------------------------------------- learned guess */

/* A small MLP that predicts density-matrix blocks from atom-pair geometry, as
 * an SCF starting point.  The paper has no counterpart (its SCF starts from
 * the core Hamiltonian, Section 3); the plain SCF is the fallback, and the
 * SCF iterations started from the guess decide the result, so a guess changes
 * iteration counts, never the converged energy.
 *   features (16 per unordered atom pair a <= b): R, u = (r_b - r_a)/R (3),
 *     u_i u_j (9), one-hot element pair (O-O, O-H, H-H); for O-H the O atom
 *     is first; on-site pairs have R = 0 and u = 0.
 *   network: 16 -> 256 -> 256 -> 325, SiLU after the first two layers; the
 *     325 outputs are three heads: O-O 15x15 (0..224), O-H 15x5 (225..299),
 *     H-H 5x5 (300..324), row-major, rows = first atom's functions.
 *   weights (float, in this order): W1[256][16], b1[256], W2[256][256],
 *     b2[256], W3[325][256], b3[325]; BF16 copies are used in the products,
 *     FP32 master copies in Adam, activations and accumulation are FP32.
 * Supported atoms: O with 15 and H with 5 contiguous Cartesian functions. */
#define HF_GUESS_FEATURES 16
#define HF_GUESS_WIDTH 256
#define HF_GUESS_OUTPUTS 325

typedef struct hf_model hf_model;

/* Number of floats in the weight vector (153,669). */
int64_t hf_model_num_params(void);

/* Create a model from host weights (hf_model_num_params floats). */
int hf_model_create(hf_ctx* ctx, const float* init_weights, hf_model** model);
void hf_model_destroy(hf_model* model);

/* Copy the FP32 master weights and/or the last gradients to host arrays
 * (either may be NULL). */
int hf_model_get_weights(hf_model* model, float* weights, float* gradients);

/* Y[n][325] = MLP(X[n][16]).  flags: HF_PTR_DEVICE for device X, Y. */
int hf_model_forward(hf_model* model, int n, const float* X, float* Y, int flags);

/* One training step on a minibatch (device pointers, HF_PTR_DEVICE
 * required): loss = (1/n) sum_i sum_j mask_ij (Y_ij - T_ij)^2, gradients by
 * backpropagation, then one Adam step (beta 0.9/0.999, eps 1e-8) with
 * learning rate lr (lr = 0 computes the gradients only).  *loss (host) may be
 * NULL. */
int hf_model_train_step(hf_model* model, int n, const float* X, const float* T, const float* mask, float lr,
                        float* loss, int flags);

/* Features of every unordered atom pair of a system.  *n_pairs =
 * n_atoms (n_atoms + 1) / 2; with X and meta NULL only the count is
 * returned.  X[n_pairs][16]; meta[n_pairs][4] = (first function of the row
 * atom, first function of the column atom, head 0/1/2, on-site flag).
 * flags: HF_PTR_DEVICE for device X/meta.  Errors: HF_E_UNSUPPORTED for
 * atoms other than the supported O and H. */
int hf_guess_features(hf_system* sys, float* X, int32_t* meta, int64_t* n_pairs, int flags);

/* Training targets of a system from a density (for example the converged
 * density of the plain SCF): for atom pair t of hf_guess_features,
 * T[t][head block] = the pair's block of P (rows = first atom's functions)
 * and mask[t][head block] = 1; every other output is 0 in both.
 *   P     [N*N] density;  T, mask  [n_pairs * 325] float outputs.
 * flags: HF_PTR_DEVICE for device P, T, mask.  Errors: HF_E_INVALID,
 * HF_E_UNSUPPORTED (atoms other than O and H), HF_E_NOMEM, HF_E_CUDA. */
int hf_guess_targets(hf_system* sys, const double* P, float* T, float* mask, int flags);

/* Options of hf_guess_train (zero-initialise, then set what differs). */
typedef struct {
    int32_t steps; /* Adam steps (required, > 0) */
    int32_t batch; /* samples per minibatch (0: 2048; at most n) */
    float lr;      /* peak learning rate (0: 1e-3) */
    int32_t pad;
    uint64_t seed; /* minibatch draws */
} hf_train_opts;

/* Minibatch training of the model on a dataset resident in device memory:
 * for step k = 0..steps-1, sample j of the minibatch is dataset row
 * SplitMix64(seed, k * batch + j) mod n (SplitMix64's output function applied
 * to seed + (i + 1) * 0x9E3779B97F4A7C15); the masked loss of
 * hf_model_train_step, its gradients, and one Adam step with learning rate
 * lr (1 + cos(pi k / steps)) / 2 (cosine decay).  The model's Adam state
 * continues from earlier calls.
 *   X [n * 16], T [n * 325], mask [n * 325]  device pointers (HF_PTR_DEVICE
 *   required), for example features and hf_guess_targets of many systems.
 *   losses  host array of `steps` minibatch losses, or NULL.
 * Errors: HF_E_INVALID (NULL argument, n <= 0, bad options, host pointers),
 * HF_E_NOMEM, HF_E_CUDA. */
int hf_guess_train(hf_model* model, int64_t n, const float* X, const float* T, const float* mask,
                   const hf_train_opts* opts, float* losses, int flags);

/* Predicted total density P[N*N]: MLP blocks placed at (a, b) and (b, a),
 * on-site blocks symmetrised, scaled so that tr(PS) = N_e.  flags:
 * HF_PTR_DEVICE.  Errors: HF_E_INVALID if the prediction is not finite or
 * tr(PS) <= 0 (the caller then falls back to the core guess). */
int hf_guess_predict(hf_model* model, hf_system* sys, double* P, int flags);

/* ------------------------------------------------- allocation-free build */

/* Largest system (basis functions) hf_fock_build_noalloc accepts. */
#define HF_NOALLOC_MAX_BF 512

/* The Fock build of hf_fock_build for callers that cannot allocate device
 * memory during the call (a process whose device memory is reserved or owned
 * by a pool that forbids cudaMalloc, or code that must not enter the
 * allocator at this point).  The paper has no counterpart: it is a property of
 * this library's interface, not of the method.
 *   P       [N*N] device pointer, total density (symmetric, finite).
 *   F       [N*N] device pointer, output H + J - K/2 (required).
 *   J, K    [N*N] device pointers, outputs (may be NULL).
 * All pointers are device pointers on the context's device; there is no host
 * path and no energy or statistics output.  The call allocates nothing: its
 * scratch (density copy, J/K accumulators, status flag; about 7.3 MB) is one
 * fixed __device__ array per device, held until the process exits and shared
 * by every call on that device.  hf_create already looked up its address
 * (and so made the driver reserve it); a context created after a device
 * reset looks it up again.  The accumulators are cleared at the start of
 * each call; calls whose device work overlaps race on the array.  A system
 * with fp32_cutoff > 0 evaluates its small quartets in FP32, as hf_fock_build
 * does without HF_FP64_ONLY.  Errors: HF_E_INVALID (NULL sys/P/F, more than
 * HF_NOALLOC_MAX_BF basis functions, P not finite or not symmetric; the
 * outputs are then left untouched), HF_E_CUDA. */
int hf_fock_build_noalloc(hf_system* sys, const double* P, double* F, double* J, double* K);

#ifdef __cplusplus
}
#endif

#endif /* HF_H */
