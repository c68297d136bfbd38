// Host-side launchers of the setup, one-electron and Fock-assembly kernels.
#pragma once
#include <cuda_runtime.h>

#include "hf_internal.h"

namespace hf {

int build_boys_tables(double* t64, float* t32, cudaStream_t s);
int launch_shell_coef(int n_sh, const int* l, const int* nprim, const int* prim0, const double* exps,
                      const double* coefs, double* cn, cudaStream_t s);
int launch_comp_norm(int n_sh, const int* l, const int* bf0, double* out, cudaStream_t s);
int launch_build_pairs(long long n_pairs, int maxpp, const int* l, const int* atom, const int* bf0, const int* nprim,
                       const int* prim0, const double* exps, const double* cn, const double* xyz, PairHdr* pairs,
                       void* p64, void* p32, int* pclass, cudaStream_t s);
int launch_class_count(long long n, const int* pclass, unsigned long long* cnt, cudaStream_t s);
int launch_class_scatter_all(long long n, const int* pclass, int X, unsigned* cursor, int* ids, cudaStream_t s);
int launch_copy_q(long long n, const double* Q, PairHdr* pairs, unsigned long long* qmax_bits, cudaStream_t s);
int launch_class_scatter_sig(long long n, const int* pclass, const double* Q, int X, double qmax, double tau,
                             unsigned* cursor, double* key, int* val, cudaStream_t s);
int bitonic_sort_desc(double* key, int* val, int n, int n_pad, cudaStream_t s);
int launch_gather_headers(int n, const int* ids, const PairHdr* pairs, PairHdr* out, cudaStream_t s);
int launch_ket_table(int n, int maxpp, long long stride, const int* ids, const PairHdr* pairs, const void* p64,
                     const void* p32, double* t64, float* t32, float* tB, cudaStream_t s);
int launch_sort_prims(long long n_pairs, const PairHdr* pairs, const double* Bprim, void* p64, void* p32, cudaStream_t s);
int launch_scan(int n, const long long* in, long long* out, cudaStream_t s);
int launch_sig_scatter(long long n_pairs, long long n_seg, const int* pclass, const double* Q,
                       const unsigned long long* qmax_bits, double tau, const size_t* seg_host, unsigned* cursor,
                       double* key, int* val, cudaStream_t s);
int launch_ket_counts_dev(int cap, const unsigned* n_bra, const double* qb, const unsigned* n_ket, const double* qk,
                          int same, double tau, double cutoff, long long* c64, long long* c32, int* kstart32,
                          cudaStream_t s);

// one-electron matrices (raw component normalisation; comp_norm applied inside)
int launch_one_electron(int n_sh, int n_atoms, int N, const int* l, const int* atom, const int* bf0,
                        const int* nprim, const int* prim0, const double* exps, const double* cn,
                        const double* xyz, const double* Z, const double* comp_norm, const double* boys64,
                        double* S, double* H, cudaStream_t s);
int launch_nuclear_repulsion(int n_atoms, const double* xyz, const double* Z, double* out, cudaStream_t s);

// Fock assembly
long long chunk_entries(long long n);
int launch_chunk_bra(int n_bra, const long long* off, long long n, int* out, cudaStream_t s);
int launch_sum_copies(int n_copies, long long nn, const double* in, double* out, int num_sms, cudaStream_t s);
int launch_axpby(long long n, const double* A, double alpha, const double* B, double* C, cudaStream_t s);
int launch_shell_block_max(int n_sh, int N, const int* l, const int* bf0, const double* P, float* dsh, cudaStream_t s);
int launch_scale_density(int N, const double* P, const double* comp_norm, double* P64, float* P32, int* bad,
                         cudaStream_t s);
int launch_assemble(int N, const double* Jt, const double* Kt, const double* comp_norm, const double* H, double* J,
                    double* K, double* F, const int* bad, cudaStream_t s);
int launch_fock_from_jk(long long n, const double* H, const double* J, const double* K, double* F, int* bad,
                        cudaStream_t s);
int launch_energy(int N, const double* P, const double* H, const double* F, double* partial, double* out,
                  cudaStream_t s);

}  // namespace hf
