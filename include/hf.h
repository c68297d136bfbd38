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

typedef struct hf_ctx hf_ctx;       /* one device + one stream + constant tables */
typedef struct hf_system hf_system; /* one molecule: basis, pairs, screening plan, 1e matrices */

/* Nuclei.  Z[n_atoms] charges; xyz[3*n_atoms] positions in bohr.  Host memory. */
typedef struct {
    int32_t n_atoms;
    const int32_t* Z;
    const double* xyz;
} hf_geometry;

/* Contracted Cartesian shells (Section 4.1's "shell": functions on one atom
 * sharing exponents).  atom[s] atom index, l[s] in 0..2, nprim[s] in 1..8,
 * exps/coefs: sum(nprim) primitive exponents and coefficients, shell after
 * shell.  Host memory. */
typedef struct {
    int32_t n_shells;
    const int32_t* atom;
    const int32_t* l;
    const int32_t* nprim;
    const double* exps;
    const double* coefs;
} hf_basis;

/* Screening and precision thresholds.
 *   schwarz_tau : skip a shell quartet when Q_ij * Q_kl < schwarz_tau
 *                 (Algorithm 1's schwartz(i,j,k,l)); 0 disables screening.
 *   fp32_cutoff : evaluate a quartet's integrals in FP32 when
 *                 Q_ij * Q_kl < fp32_cutoff (accumulation stays FP64);
 *                 0 keeps every quartet in FP64.
 *   prim_tau    : reserved, must be 0. */
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
 * tables on the device.  Errors: HF_E_INVALID (ctx NULL),
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
 * range, non-positive exponent, NaN), HF_E_UNSUPPORTED (l > 2,
 * nprim > 8, prim_tau != 0), HF_E_NOMEM, HF_E_CUDA. */
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
 * flags: HF_PTR_DEVICE (P, F, J, K are device pointers), HF_TIMING.
 * Errors: HF_E_INVALID (NULL sys/P, P not finite or not symmetric),
 * HF_E_NOMEM, HF_E_CUDA. */
int hf_fock_build(hf_system* sys, const double* P, double* F, double* J, double* K, double* E_elec, hf_stats* stats,
                  int flags);

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
 * by every call on that device.  The accumulators are cleared at the start of
 * each call; calls whose device work overlaps race on the array.  The first
 * call on a device looks the array's address up once; make it before any
 * stream capture.  Errors: HF_E_INVALID (NULL sys/P/F, more than
 * HF_NOALLOC_MAX_BF basis functions, P not finite or not symmetric),
 * HF_E_CUDA. */
int hf_fock_build_noalloc(hf_system* sys, const double* P, double* F, double* J, double* K);

#ifdef __cplusplus
}
#endif

#endif /* HF_H */
