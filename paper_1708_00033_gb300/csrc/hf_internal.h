// Internal declarations of the GB300 direct-SCF Fock-build library.
// Not part of the C-ABI (that is include/hf.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/hf.h"

namespace hf {

constexpr int kMaxL = 2;
constexpr int kNumPairClasses = 6;  // ss ps pp ds dp dd
constexpr int kNumClasses = 21;     // (X|Y), X >= Y
constexpr int kChunkShift = 10;      // quartets per entry of the bra lookup tables: 1024
constexpr int kMaxPrim = 8;         // primitives per shell accepted by the library

// One significant shell pair, oriented so that l_A >= l_B.
struct PairHdr {
    int A, B;          // shell ids
    int bfA, bfB;      // first basis function of shells A and B
    int prim0, nprim;  // primitive-pair records [prim0, prim0 + nprim)
    double ABx, ABy, ABz;
    double Q;          // Cauchy-Schwarz bound sqrt(max |(mu nu|mu nu)|)
    float ABfx, ABfy, ABfz;  // A - B in FP32 (the FP32 kernels' horizontal step uses no FP64 instruction)
};

struct EriArgs {
    const PairHdr* pairs;
    const void* prims64;  // PrimPair<double>[]
    const void* prims32;  // PrimPair<float>[]
    const int* bra;       // bra pair ids (one class, sorted by Q descending)
    const int* ket;       // ket pair ids
    const long long* offsets;  // [n_bra + 1] exclusive prefix of quartets per bra
    const int* kstart;         // [n_bra] first ket of each bra (nullptr: 0)
    int n_bra;
    int same;                  // bra and ket lists are the same list
    long long n_quartets;
    int N;
    const double* P64;  // density in the library's raw component normalisation
    const float* P32;
    double* Jt;
    double* Kt;
    const double* boys64;
    const float* boys32;
    double prim_tau;                  // skip primitive quartets with B_ab * B_cd < prim_tau
    unsigned long long* prim_count;   // evaluated primitive quartets (nullptr: not counted)
    long long q_begin;                // first quartet of this launch (quartets [q_begin, n_quartets))
    const float* dsh;                 // [n_sh x n_sh] max |P| per shell block (nullptr: no density screening)
    int n_sh;
    float dtau;                       // density-weighted screening threshold
    const int* chunk;                 // [c] bra of quartet min(c << kChunkShift, n_quartets_all - 1)
                                      // (nullptr: each quartet's bra by binary search over all bras)
    int n_copies;                     // > 1: block b accumulates into copy b % n_copies of Jt / Kt
    long long copy_stride;            // doubles between copies
    const int* bad;                   // density-check flag: the kernel does nothing when *bad != 0
    const void* kt;                   // ket table of the launch's ket class and precision (field-major records
                                      // in class-list order, see KetSoa): read by the FP32 and Rys kernels; the
                                      // FP64 Obara-Saika kernels read each pair's own records
    const float* ktB;                 // primitive-pair bounds of the ket table
    long long kstride;                // kets per field row of the ket table
    const PairHdr* bhdr;              // headers of the bra list in list order (bhdr[b] = pairs[bra[b]])
    const PairHdr* khdr;              // headers of the ket list in list order (khdr[k] = pairs[ket[k]])
    int sort_work;                    // 1: each warp runs its window of quartets sorted by staircase length
};

struct SchwarzArgs {
    const PairHdr* pairs;
    const void* prims64;  // PrimPair<double>[]
    const int* ids;       // pair ids of one diagonal class
    int n;
    double* Q;            // [pair id] output bound
    const double* boys64;
    double* Bprim;        // [primitive pair] output bound of each primitive pair
    int items;            // threads per pair: 1 + the largest primitive-pair count
};

// One molecule's view of one class in a batched build.
struct MolClass {
    const PairHdr* pairs;
    const void* prims64;
    const int* bra;
    const int* ket;
    const long long* offsets;  // [n_bra + 1]
    int n_bra;
    int same;
    int N;
    int pad;
    const double* P64;
    double* Jt;
    double* Kt;
};

struct BatchArgs {
    const MolClass* mols;        // [n_mol]
    const long long* mol_off;    // [n_mol + 1] exclusive prefix of this class's quartets per molecule
    int n_mol;
    int chunk;                   // quartets per work-queue grab (per warp)
    long long n_total;
    unsigned long long* counter; // work-queue head, zero at launch
    double prim_tau;
    const double* boys64;
};

struct EriClassEntry {
    int X, Y, L;
    int prim_flops;  // per primitive quartet (setup + Boys + VRR + accumulation)
    int cont_flops;  // per contracted quartet (HRR + digestion)
    void (*launch)(const EriArgs&, int use_f32, int grid, int block, cudaStream_t, int lanes);
    void (*launch_schwarz)(const SchwarzArgs&, int block, cudaStream_t);
    const char* name;
    void (*launch_batch)(const BatchArgs&, int grid, int block, cudaStream_t);
    size_t (*local_bytes)();  // largest per-thread local memory of the class's kernels
    int lanes;                // lanes that share one shell quartet in the ERI kernels
    // Rys-quadrature variant (classes with L >= 6; nullptr otherwise): FP64 launches with ket tables
    void (*launch_rys)(const EriArgs&, int use_f32, int grid, int block, cudaStream_t, int lanes);
    int prim_flops_rys;       // per primitive quartet (setup + roots + 2D recurrences + accumulation)
    size_t (*local_bytes_rys)();
    int rys_default;          // 1: FP64 launches use the Rys variant unless HF_OBARA_SAIKA is given
};
extern const EriClassEntry kEriClasses[kNumClasses];

// Whether the FP64 launches of class ci take the Rys variant under these build flags: HF_RYS for every
// class that has one, HF_OBARA_SAIKA for none, else the class's default.
inline bool class_uses_rys(int ci, int flags)
{
    if (!kEriClasses[ci].launch_rys || (flags & HF_OBARA_SAIKA)) return false;
    return (flags & HF_RYS) || kEriClasses[ci].rys_default;
}

// Launches the ERI class kernels of one build: for every class and precision, the quartets
// [n shard / n_shards, n (shard + 1) / n_shards) of its n screened quartets (shard 0 of 1 is the
// whole build).  `a` carries the fields common to every launch (density, accumulators, tables,
// screening and flag pointers); the per-class fields are filled here.  flags: HF_FP64_ONLY.
// ev (nullable): events 4 c + 2 prec and 4 c + 2 prec + 1 are recorded around each class launch;
// prim_count (nullable): 2 c + prec counts the evaluated primitive quartets of each launch.
int launch_eri_classes(hf_system* S, EriArgs a, int shard, int n_shards, int flags, cudaEvent_t* ev,
                       unsigned long long* prim_count);

// Device address of the allocation-free build's fixed scratch on the current device (noalloc.cu).
int noalloc_scratch_address(void** out);

// ---------------------------------------------------------------- errors --
struct Status {
    int code = HF_OK;
    std::string msg;
};
void set_error(int code, const std::string& msg);
int cuda_status(cudaError_t e, const char* what);

#define HF_CUDA(call)                                          \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_status(e_, #call);  \
    } while (0)

// -------------------------------------------------- device buffer helper --
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    bool owned = true;
    int alloc(size_t n);
    void release();
    // non-owning view of part of another buffer (an arena)
    void view(void* ptr, size_t n)
    {
        release();
        p = ptr;
        bytes = n;
        owned = false;
    }
    template <typename T>
    T* as() const { return (T*)p; }
    ~DevBuf() { release(); }
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
};

}  // namespace hf

// ----------------------------------------------------------- C-ABI types --
struct hf_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    hf::DevBuf boys64, boys32;  // Boys Taylor tables
    cudaEvent_t ev[4 * hf::kNumClasses + 4] = {};
    bool events_ready = false;
    int n_systems = 0;            // live systems created on this context
    bool destroy_pending = false;  // hf_destroy was called while systems were alive
    void* noalloc_scratch = nullptr;  // device address of hf_fock_build_noalloc's fixed scratch
};

struct hf_system {
    hf_ctx* ctx = nullptr;
    int device = 0;               // copies of the context's device and stream, so that
    cudaStream_t stream = nullptr;  // destruction never needs the context
    int n_atoms = 0, n_shells = 0, n_bf = 0, n_electrons = 0;
    double E_nn = 0.0;
    hf_thresholds th{};
    // shells (device)
    hf::DevBuf sh_l, sh_atom, sh_bf0, sh_nprim, sh_prim0, sh_exp, sh_coef, atom_xyz, atom_Z;
    hf::DevBuf comp_norm;  // [n_bf] Cartesian component factor
    // pairs
    int n_pairs_all = 0, n_prim_pairs = 0;
    hf::DevBuf pairs, prims64, prims32, pair_class;
    int class_count[hf::kNumPairClasses] = {};
    hf::DevBuf class_ids[hf::kNumPairClasses];  // sorted significant pair ids
    double Qmax = 0.0;
    // quartet schedule per class
    struct ClassPlan {
        hf::DevBuf offsets64, offsets32, kstart32;
        hf::DevBuf chunk64, chunk32;  // bra of every 2^kChunkShift-th quartet (see EriArgs::chunk)
        long long n64 = 0, n32 = 0;
        long long n_unscreened = 0;
    } plan[hf::kNumClasses];
    // matrices (device)
    hf::DevBuf S, H, P64, P32, Jt, Kt, J, K, F, Ebuf, host_stage;
    int64_t quartets_total = 0;
    // scratch
    hf::DevBuf class_q[hf::kNumPairClasses];  // sorted bounds of class_ids
    hf::DevBuf Qall, counts, staging_P, staging_out, bad, Bprim, prim_count;
    hf::DevBuf arena_in, arena_mat, arena_sched;  // owners of the views above
    hf::DevBuf dsh;                                // density block maxima for density-weighted screening
    // ket tables: per pair class, the significant pairs' primitive-pair records in class-list order and
    // field-major (9 maxpp rows of FP64 fields, 9 maxpp rows of FP32 fields, maxpp rows of bounds)
    hf::DevBuf ket_tab[hf::kNumPairClasses];
    hf::DevBuf class_hdr[hf::kNumPairClasses];  // pair headers of each class list, in list order
    long long ket_stride[hf::kNumPairClasses] = {};
    int fock_copies = 1;                           // accumulator copies of Jt / Kt (1: one shared copy)
    hf::DevBuf copies;                             // [2][fock_copies][N*N] when fock_copies > 1
    int maxpp = 0;
    // host copies used by the learned guess: nuclear charges, first basis
    // function and function count of each atom (-1 if its shells are not contiguous)
    std::vector<int> Z_h, atom_bf0_h, atom_nbf_h;
};
