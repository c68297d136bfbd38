// SCF driver (Section 3 of the paper, Eq. FC = eSC): symmetric (Lowdin)
// orthogonalisation X = S^-1/2 (canonical when an overlap eigenvalue is below
// 1e-8), core-Hamiltonian guess, then repeat
//   F = F(P) (hf_fock_build)  ->  Pulay DIIS on e = FPS - SPF  ->
//   F' = X^T F X, Jacobi eigenpairs  ->  C_occ = X C'_occ  ->  P = 2 C_occ C_occ^T
// until |dE| < e_tol and RMS(dP) < d_tol.  Every matrix step runs on the
// device; per iteration only scalars (E, RMS dP, DIIS status) reach the host.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <string>
#include <vector>

#include "hf_internal.h"
#include "linalg.cuh"
#include "setup.cuh"

namespace hf {
namespace {

int scf_fail(int code, const std::string& msg)
{
    set_error(code, msg);
    return code;
}

#define S_TRY(x)                       \
    do {                               \
        int rc_ = (x);                 \
        if (rc_ != HF_OK) return rc_;  \
    } while (0)
#define S_K(x)                                                               \
    do {                                                                     \
        if ((x) != 0) return cuda_status(cudaGetLastError(), "scf: " #x);   \
    } while (0)

struct ScopedDevice {
    int prev = -1;
    explicit ScopedDevice(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~ScopedDevice()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Eigen-decomposition with its own workspace.
struct Eigh {
    DevBuf work, iwork;
    int n = 0;
    int init(int n_)
    {
        n = n_;
        S_TRY(work.alloc(jacobi_work_doubles(n) * sizeof(double)));
        S_TRY(iwork.alloc(jacobi_work_ints(n) * sizeof(int)));
        return HF_OK;
    }
    int run(const double* A, double* w, double* V, int ncols, int* sweeps, cudaStream_t s)
    {
        int sw = 0;
        const int rc = jacobi_eigh(n, A, w, V, ncols, work.as<double>(), iwork.as<int>(), 60, 1e-14, &sw, s);
        if (sweeps) *sweeps += sw;
        if (rc < 0) return cuda_status(cudaGetLastError(), "jacobi_eigh");
        if (rc > 0) return scf_fail(HF_E_NOCONV, "Jacobi eigensolver did not converge in 60 sweeps");
        return HF_OK;
    }
};

}  // namespace
}  // namespace hf

using namespace hf;

extern "C" int hf_eigh(hf_ctx* ctx, int n, const double* A, double* w, double* V, int flags)
{
    if (!ctx || !A || !w || !V || n <= 0) return scf_fail(HF_E_INVALID, "hf_eigh: NULL argument or n <= 0");
    ScopedDevice g(ctx->device);
    cudaStream_t st = ctx->stream;
    const bool dev = (flags & HF_PTR_DEVICE) != 0;
    const size_t nn = (size_t)n * n;
    DevBuf dA, dw, dV;
    const double* pA = A;
    double* pw = w;
    double* pV = V;
    if (!dev) {
        S_TRY(dA.alloc(nn * sizeof(double)));
        S_TRY(dw.alloc(n * sizeof(double)));
        S_TRY(dV.alloc(nn * sizeof(double)));
        HF_CUDA(cudaMemcpyAsync(dA.p, A, nn * sizeof(double), cudaMemcpyHostToDevice, st));
        pA = dA.as<double>();
        pw = dw.as<double>();
        pV = dV.as<double>();
    }
    Eigh e;
    S_TRY(e.init(n));
    S_TRY(e.run(pA, pw, pV, n, nullptr, st));
    if (!dev) {
        HF_CUDA(cudaMemcpyAsync(w, pw, n * sizeof(double), cudaMemcpyDeviceToHost, st));
        HF_CUDA(cudaMemcpyAsync(V, pV, nn * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    HF_CUDA(cudaStreamSynchronize(st));
    return HF_OK;
}

extern "C" int hf_scf_run(hf_system* S, const hf_scf_opts* opts_in, const double* P_guess, double* P_out,
                          double* eps_out, double* energies, hf_scf_result* res, int flags)
{
    if (!S || !res) return scf_fail(HF_E_INVALID, "hf_scf_run: NULL system or result");
    hf_scf_opts o;
    memset(&o, 0, sizeof(o));
    o.max_iter = 100;
    o.e_tol = 1e-9;
    o.d_tol = 1e-6;
    o.diis_size = 8;
    if (opts_in) {
        o = *opts_in;
        if (o.max_iter == 0) o.max_iter = 100;
        if (o.e_tol == 0.0) o.e_tol = 1e-9;
        if (o.d_tol == 0.0) o.d_tol = 1e-6;
        if (o.diis_size == 0 && !o.diis_off) o.diis_size = 8;
        if (o.diis_off) o.diis_size = 0;
        if (o.mixed_switch == 0.0) o.mixed_switch = 1e-5;
        if (o.rebuild_every <= 0) o.rebuild_every = 8;
        if (o.incremental_switch == 0.0) o.incremental_switch = 1e-5;
    }
    if (!opts_in) o.rebuild_every = 8;
    if (!opts_in) o.incremental_switch = 1e-5;
    if (!opts_in) o.mixed_switch = 1e-5;
    bool mixed = S->th.fp32_cutoff > 0.0;
    const int N = S->n_bf;
    const int n_occ = o.n_occ > 0 ? o.n_occ : S->n_electrons / 2;
    if (n_occ <= 0 || n_occ > N) return scf_fail(HF_E_INVALID, "hf_scf_run: occupied orbital count out of range");
    if (o.max_iter <= 0 || o.diis_size < 0 || o.diis_size > 16 || !(o.e_tol > 0) || !(o.d_tol > 0))
        return scf_fail(HF_E_INVALID, "hf_scf_run: bad options");
    ScopedDevice g(S->device);
    cudaStream_t st = S->stream;
    const bool dev = (flags & HF_PTR_DEVICE) != 0;
    const size_t NN = (size_t)N * N;
    const double t0 = now_s();
    memset(res, 0, sizeof(*res));
    res->E_nn = S->E_nn;

    // ------------------------------------------------------ orthogonaliser
    DevBuf sv, U, Us, X, T1, T2, Fp, Vp, Cocc, P, Pn, Fcur, Fuse, err, part, scal, coef, stat, ptrs;
    S_TRY(sv.alloc(N * sizeof(double)));
    S_TRY(U.alloc(NN * sizeof(double)));
    S_TRY(Us.alloc(NN * sizeof(double)));
    S_TRY(X.alloc(NN * sizeof(double)));
    S_TRY(T1.alloc(NN * sizeof(double)));
    S_TRY(T2.alloc(NN * sizeof(double)));
    S_TRY(Fp.alloc(NN * sizeof(double)));
    S_TRY(Vp.alloc(NN * sizeof(double)));
    S_TRY(Cocc.alloc((size_t)N * n_occ * sizeof(double)));
    S_TRY(P.alloc(NN * sizeof(double)));
    S_TRY(Pn.alloc(NN * sizeof(double)));
    S_TRY(Fuse.alloc(NN * sizeof(double)));
    S_TRY(part.alloc(4096 * sizeof(double)));
    S_TRY(scal.alloc(64 * sizeof(double)));
    S_TRY(coef.alloc(32 * sizeof(double)));
    S_TRY(stat.alloc(sizeof(int)));
    S_TRY(ptrs.alloc(64 * sizeof(void*)));
    const int m_diis = std::max(1, o.diis_size);
    std::vector<DevBuf> Fh(m_diis), Eh(m_diis);
    for (int k = 0; k < m_diis; k++) {
        S_TRY(Fh[k].alloc(NN * sizeof(double)));
        S_TRY(Eh[k].alloc(NN * sizeof(double)));
    }
    Eigh eig;
    S_TRY(eig.init(N));
    int sweeps = 0;
    double t_diag = 0.0, t_fock = 0.0;
    double td = now_s();
    S_TRY(eig.run(S->S.as<double>(), sv.as<double>(), U.as<double>(), N, &sweeps, st));
    std::vector<double> s_host(N);
    HF_CUDA(cudaMemcpyAsync(s_host.data(), sv.p, N * sizeof(double), cudaMemcpyDeviceToHost, st));
    HF_CUDA(cudaStreamSynchronize(st));
    t_diag += now_s() - td;
    int drop = 0;
    while (drop < N && s_host[drop] < 1e-8) drop++;
    if (drop == N) return scf_fail(HF_E_INVALID, "hf_scf_run: overlap matrix has no eigenvalue above 1e-8");
    const int nx = N - drop;
    if (nx < n_occ) return scf_fail(HF_E_INVALID, "hf_scf_run: fewer independent functions than occupied orbitals");
    res->n_kept = nx;
    res->s_min = s_host[0];
    S_K(scale_cols(N, N, U.as<double>(), sv.as<double>(), -0.5, 1e-8, Us.as<double>(), st));
    const double* Xp;
    int ldx;
    if (drop == 0) {  // Lowdin: X = U s^-1/2 U^T
        S_K(gemm(N, N, N, 1.0, Us.as<double>(), N, false, U.as<double>(), N, true, 0.0, X.as<double>(), N, st));
        Xp = X.as<double>();
        ldx = N;
    } else {  // canonical: X = U[:, drop:] s^-1/2
        Xp = Us.as<double>() + drop;
        ldx = N;
    }
    DevBuf Vprev, Vj, Fw;
    S_TRY(Vprev.alloc(NN * sizeof(double)));
    S_TRY(Vj.alloc(NN * sizeof(double)));
    S_TRY(Fw.alloc(NN * sizeof(double)));
    bool have_prev = false;
    auto diagonalise = [&](const double* Fm, double* Pout, double* eps) -> int {
        // F' = X^T F X (nx x nx), eigenpairs, C_occ = X C'_occ, P = 2 C_occ C_occ^T.  After the
        // first iteration F' is rotated into the previous eigenvectors' basis, where it is nearly
        // diagonal, so the Jacobi sweeps start close to convergence (V = V_prev V_jacobi).
        double tt = now_s();
        if (gemm(N, nx, N, 1.0, Fm, N, false, Xp, ldx, false, 0.0, T1.as<double>(), nx, st)) return -1;
        if (gemm(nx, nx, N, 1.0, Xp, ldx, true, T1.as<double>(), nx, false, 0.0, Fp.as<double>(), nx, st)) return -1;
        int rc = HF_OK;
        Eigh* e = &eig;
        Eigh e2;
        if (nx != N) {
            rc = e2.init(nx);
            if (rc != HF_OK) return rc;
            e = &e2;
        }
        if (have_prev) {
            if (gemm(nx, nx, nx, 1.0, Fp.as<double>(), nx, false, Vprev.as<double>(), nx, false, 0.0, T1.as<double>(),
                     nx, st))
                return -1;
            if (gemm(nx, nx, nx, 1.0, Vprev.as<double>(), nx, true, T1.as<double>(), nx, false, 0.0, Fw.as<double>(),
                     nx, st))
                return -1;
            rc = e->run(Fw.as<double>(), eps, Vj.as<double>(), nx, &sweeps, st);
            if (rc != HF_OK) return rc;
            if (gemm(nx, nx, nx, 1.0, Vprev.as<double>(), nx, false, Vj.as<double>(), nx, false, 0.0, Vp.as<double>(),
                     nx, st))
                return -1;
        } else {
            rc = e->run(Fp.as<double>(), eps, Vp.as<double>(), nx, &sweeps, st);
            if (rc != HF_OK) return rc;
        }
        if (cudaMemcpyAsync(Vprev.p, Vp.p, (size_t)nx * nx * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return -1;
        have_prev = true;
        // C_occ = X[:, :nx] * V[:, :n_occ]  (V is nx x nx, row-major, first n_occ columns)
        if (gemm(N, n_occ, nx, 1.0, Xp, ldx, false, Vp.as<double>(), nx, false, 0.0, Cocc.as<double>(), n_occ, st))
            return -1;
        if (gemm(N, N, n_occ, 2.0, Cocc.as<double>(), n_occ, false, Cocc.as<double>(), n_occ, true, 0.0, Pout, N, st))
            return -1;
        cudaStreamSynchronize(st);
        t_diag += now_s() - tt;
        return HF_OK;
    };
    DevBuf epsd;
    S_TRY(epsd.alloc(N * sizeof(double)));
    // ------------------------------------------------------------- guess
    if (P_guess) {
        HF_CUDA(cudaMemcpyAsync(P.p, P_guess, NN * sizeof(double), dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                st));
    } else {
        int rc = diagonalise(S->H.as<double>(), P.as<double>(), epsd.as<double>());
        if (rc < 0) return cuda_status(cudaGetLastError(), "scf: core-Hamiltonian guess");
        if (rc != HF_OK) return rc;
    }
    // --------------------------------------------------------- iterations
    double E_old = 0.0, E = 0.0, dP = 0.0;
    int it = 0, converged = 0, nh = 0, head = 0;
    DevBuf Jacc, Kacc, Pref, Dd, Jd, Kd;
    if (o.incremental) {
        S_TRY(Jacc.alloc(NN * sizeof(double)));
        S_TRY(Kacc.alloc(NN * sizeof(double)));
        S_TRY(Pref.alloc(NN * sizeof(double)));
        S_TRY(Dd.alloc(NN * sizeof(double)));
        S_TRY(Jd.alloc(NN * sizeof(double)));
        S_TRY(Kd.alloc(NN * sizeof(double)));
    }
    int since_full = 0;
    bool force_full = true;
    bool inc_on = o.incremental != 0;  // cleared near convergence: the rest are full builds
    std::vector<const double*> fptr(m_diis), eptr(m_diis);
    for (it = 1; it <= o.max_iter; it++) {
        double E_el = 0.0;
        const double tf = now_s();
        double* Fslot = Fh[head].as<double>();
        const int pflags = HF_PTR_DEVICE | (mixed ? 0 : HF_FP64_ONLY);
        bool full = true;
        int rc;
        if (!o.incremental) {
            rc = hf_fock_build(S, P.as<double>(), Fslot, nullptr, nullptr, &E_el, nullptr, pflags);
            if (rc != HF_OK) return rc;
        } else {
            full = !inc_on || force_full || since_full >= o.rebuild_every;
            if (full) {  // J, K of the full density
                rc = hf_fock_build_partial(S, P.as<double>(), 0, 1, Jacc.as<double>(), Kacc.as<double>(), pflags);
                if (rc != HF_OK) return rc;
                since_full = 0;
                res->full_builds++;
            } else {  // J, K += J, K of the density change, density-weighted screening
                S_K(launch_axpby((long long)NN, P.as<double>(), -1.0, Pref.as<double>(), Dd.as<double>(), st));
                rc = hf_fock_build_partial(S, Dd.as<double>(), 0, 1, Jd.as<double>(), Kd.as<double>(),
                                           pflags | HF_DENSITY_SCREEN);
                if (rc != HF_OK) return rc;
                S_K(launch_axpby((long long)NN, Jacc.as<double>(), 1.0, Jd.as<double>(), Jacc.as<double>(), st));
                S_K(launch_axpby((long long)NN, Kacc.as<double>(), 1.0, Kd.as<double>(), Kacc.as<double>(), st));
                since_full++;
            }
            force_full = false;
            HF_CUDA(cudaMemcpyAsync(Pref.p, P.p, NN * sizeof(double), cudaMemcpyDeviceToDevice, st));
            // F = H + J - K/2 and E_elec = 1/2 sum P (H + F)
            S_K(launch_axpby((long long)NN, S->H.as<double>(), 1.0, Jacc.as<double>(), Fslot, st));
            S_K(launch_axpby((long long)NN, Fslot, -0.5, Kacc.as<double>(), Fslot, st));
            S_K(launch_energy(N, P.as<double>(), S->H.as<double>(), Fslot, part.as<double>(), scal.as<double>() + 8, st));
            HF_CUDA(cudaMemcpyAsync(&E_el, scal.as<double>() + 8, sizeof(double), cudaMemcpyDeviceToHost, st));
            HF_CUDA(cudaStreamSynchronize(st));
        }
        t_fock += now_s() - tf;
        E = E_el + S->E_nn;
        if (energies) energies[it - 1] = E;
        if (mixed) res->mixed_iterations++;
        // DIIS error e = FPS - SPF = T - T^T with T = F P S
        S_K(gemm(N, N, N, 1.0, Fslot, N, false, P.as<double>(), N, false, 0.0, T1.as<double>(), N, st));
        S_K(gemm(N, N, N, 1.0, T1.as<double>(), N, false, S->S.as<double>(), N, false, 0.0, T2.as<double>(), N, st));
        S_K(antisym(N, T2.as<double>(), Eh[head].as<double>(), st));
        nh = std::min(nh + 1, m_diis);
        head = (head + 1) % m_diis;
        const double* Fm = Fslot;
        if (o.diis_size >= 2 && nh >= 2) {
            // history slots, oldest first
            for (int k = 0; k < nh; k++) {
                const int slot = (head - nh + k + m_diis) % m_diis;
                fptr[k] = Fh[slot].as<double>();
                eptr[k] = Eh[slot].as<double>();
            }
            HF_CUDA(cudaMemcpyAsync(ptrs.p, eptr.data(), nh * sizeof(void*), cudaMemcpyHostToDevice, st));
            HF_CUDA(cudaMemcpyAsync((void**)ptrs.p + 32, fptr.data(), nh * sizeof(void*), cudaMemcpyHostToDevice, st));
            DevBuf Bm;
            S_TRY(Bm.alloc(nh * nh * sizeof(double)));
            for (int r = 0; r < nh; r++)
                S_K(dots((long long)NN, eptr[r], (const double* const*)ptrs.p, nh, part.as<double>(),
                         Bm.as<double>() + r * nh, st));
            S_K(diis_solve(nh, Bm.as<double>(), coef.as<double>(), stat.as<int>(), st));
            int status = 0;
            HF_CUDA(cudaMemcpyAsync(&status, stat.p, sizeof(int), cudaMemcpyDeviceToHost, st));
            HF_CUDA(cudaStreamSynchronize(st));
            if (status == 0) {
                S_K(lincomb((long long)NN, nh, (const double* const*)((void**)ptrs.p + 32), coef.as<double>(),
                            Fuse.as<double>(), st));
                Fm = Fuse.as<double>();
            }
        }
        rc = diagonalise(Fm, Pn.as<double>(), epsd.as<double>());
        if (rc < 0) return cuda_status(cudaGetLastError(), "scf: diagonalisation");
        if (rc != HF_OK) return rc;
        S_K(rms_diff((long long)NN, Pn.as<double>(), P.as<double>(), part.as<double>(), scal.as<double>(), st));
        HF_CUDA(cudaMemcpyAsync(&dP, scal.p, sizeof(double), cudaMemcpyDeviceToHost, st));
        HF_CUDA(cudaStreamSynchronize(st));
        res->last_dE = it > 1 ? fabs(E - E_old) : INFINITY;
        res->last_dP = dP;
        if (!mixed && it > 1 && fabs(E - E_old) < o.e_tol && dP < o.d_tol) {
            if (full) {
                converged = 1;
                break;
            }
            // the accumulated J, K carry the screening error of every difference build since the last
            // full one: finish with builds from the full density, as the plain method would
            inc_on = false;
        }
        if (inc_on && it > 1 && fabs(E - E_old) < o.incremental_switch) {
            // near convergence the difference builds' accumulated screening error (a Fock matrix that
            // depends on the path, not only on P) would stall DIIS: full builds from here on, and the
            // Fock matrices of the incremental phase leave the DIIS history
            inc_on = false;
            nh = 0;
        }
        if (mixed && it > 1 && fabs(E - E_old) < o.mixed_switch) {
            mixed = false;  // switch to FP64-only builds; the mixed-phase Fock matrices leave the DIIS history
            nh = 0;
            force_full = true;  // and the accumulated J, K are rebuilt in FP64
        }
        E_old = E;
        std::swap(P.p, Pn.p);
    }
    if (it > o.max_iter) it = o.max_iter;
    res->energy = E;
    res->iterations = it;
    if (!o.incremental) res->full_builds = it;
    res->converged = converged;
    res->jacobi_sweeps = sweeps;
    res->seconds_fock = t_fock;
    res->seconds_diag = t_diag;
    const cudaMemcpyKind out_kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (P_out) HF_CUDA(cudaMemcpyAsync(P_out, P.p, NN * sizeof(double), out_kind, st));
    if (eps_out) HF_CUDA(cudaMemcpyAsync(eps_out, epsd.p, nx * sizeof(double), out_kind, st));
    HF_CUDA(cudaStreamSynchronize(st));
    res->seconds_total = now_s() - t0;
    if (!converged) return scf_fail(HF_E_NOCONV, "hf_scf_run: not converged in max_iter iterations");
    return HF_OK;
}
