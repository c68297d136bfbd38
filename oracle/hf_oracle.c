/*
 * CPU FP64 oracle for the direct-SCF Fock build.
 *
 * TEST INFRASTRUCTURE ONLY: this file is compiled and called by tests/,
 * __graft_entry__.smoke() and bench.py's CPU-baseline leg, never by the
 * product path.  It shares no code, tables or helpers with the CUDA library.
 *
 * What it computes (closed-shell RHF, Section 3 of the paper, Eq. FC = eSC):
 *   - contracted Cartesian Gaussian basis, each component rescaled so that
 *     S_mu,mu = 1;
 *   - one-electron matrices S, T, V and the nuclear repulsion E_nn;
 *   - electron-repulsion integrals (mu nu|lam sig) by the McMurchie-Davidson
 *     Hermite expansion (Helgaker, Jorgensen, Olsen, ch. 9): Hermite
 *     coefficients E^{ij}_t by their two-term recurrences, Hermite Coulomb
 *     integrals R^n_{tuv} by their recurrences from Boys functions;
 *   - Boys function F_m(T) by its convergent series for T < 40 followed by
 *     downward recursion, and by the erf limit plus upward recursion above;
 *   - J_mu nu = sum P_lam sig (mu nu|lam sig), K_mu nu = sum P_lam sig
 *     (mu lam|nu sig), either literally over all ordered indices from a
 *     stored integral table, or by streaming the symmetry-unique shell
 *     quartets of Algorithm 1 (i >= j, k <= i, l up to the canonical limit)
 *     and applying the six updates of Eq. 1a-1f with the degeneracy weights
 *     the paper leaves implicit;
 *   - Cauchy-Schwarz shell-pair bounds Q_ij = sqrt(max |(mu nu|mu nu)|).
 * Screening in the unique-quartet path is optional (tau = 0 disables it).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXL 2
#define OR_MAXPRIM 16
#define OR_MAXCOMP 6
#define OR_LTOT (4 * OR_MAXL)
#define OR_PI 3.14159265358979323846

typedef struct {
    int l, nprim, ncomp, bf0, atom;
    double A[3];
    double alpha[OR_MAXPRIM];
    double d[OR_MAXCOMP][OR_MAXPRIM]; /* final coefficient per component per primitive */
    int pw[OR_MAXCOMP][3];            /* Cartesian powers of each component */
} or_shell;

typedef struct {
    int n_atoms, n_shells, n_bf;
    double* Z;
    double* xyz;
    or_shell* sh;
} or_ctx;

/* ---------------------------------------------------------------- Boys -- */
/* F_m(T) = int_0^1 t^{2m} exp(-T t^2) dt for m = 0..mmax. */
void or_boys(int mmax, double T, double* F)
{
    if (T < 40.0) {
        /* F_m(T) = exp(-T) sum_k (2T)^k / ((2m+1)(2m+3)...(2m+2k+1)) */
        double term = 1.0 / (2 * mmax + 1), sum = term;
        for (int k = 1; k < 2000; k++) {
            term *= 2.0 * T / (2 * mmax + 2 * k + 1);
            sum += term;
            if (term < 1e-18 * sum) break;
        }
        double e = exp(-T);
        F[mmax] = e * sum;
        for (int m = mmax - 1; m >= 0; m--) F[m] = (2.0 * T * F[m + 1] + e) / (2 * m + 1);
    } else {
        double e = exp(-T);
        F[0] = 0.5 * sqrt(OR_PI / T) * erf(sqrt(T));
        for (int m = 0; m < mmax; m++) F[m + 1] = ((2 * m + 1) * F[m] - e) / (2.0 * T);
    }
}

/* ------------------------------------------------- Hermite expansions -- */
#define EI 5  /* i, j up to 4 (kinetic energy needs l+2) */
#define ET 10
typedef double etab[EI][EI][ET];

/* E^{ij}_t for one Cartesian direction, i <= imax, j <= jmax. */
static void hermite_E(int imax, int jmax, double a, double b, double Ax, double Bx, etab E)
{
    double p = a + b, mu = a * b / p, Px = (a * Ax + b * Bx) / p;
    double XPA = Px - Ax, XPB = Px - Bx, XAB = Ax - Bx, h = 1.0 / (2.0 * p);
    memset(E, 0, sizeof(etab));
    E[0][0][0] = exp(-mu * XAB * XAB);
    for (int i = 0; i <= imax; i++) {
        for (int j = 0; j <= jmax; j++) {
            if (i == 0 && j == 0) continue;
            for (int t = 0; t <= i + j; t++) {
                if (i > 0) {
                    E[i][j][t] = (t > 0 ? h * E[i - 1][j][t - 1] : 0.0) + XPA * E[i - 1][j][t]
                               + (t + 1) * E[i - 1][j][t + 1];
                } else {
                    E[i][j][t] = (t > 0 ? h * E[i][j - 1][t - 1] : 0.0) + XPB * E[i][j - 1][t]
                               + (t + 1) * E[i][j - 1][t + 1];
                }
            }
        }
    }
}

#define RN (OR_LTOT + 1)
/* R^0_{tuv}(alpha, X, Y, Z) for t+u+v <= L, stored R[t][u][v]. */
static void hermite_R(int L, double alpha, double X, double Y, double Z, double R[RN][RN][RN])
{
    static __thread double Rn[RN][RN][RN][RN];
    double F[RN + 1];
    or_boys(L, alpha * (X * X + Y * Y + Z * Z), F);
    double f = 1.0;
    for (int n = 0; n <= L; n++) {
        Rn[n][0][0][0] = f * F[n];
        f *= -2.0 * alpha;
    }
    for (int n = L - 1; n >= 0; n--) {
        int top = L - n;
        for (int t = 0; t <= top; t++)
            for (int u = 0; u + t <= top; u++)
                for (int v = 0; v + u + t <= top; v++) {
                    if (t + u + v == 0) continue;
                    double r;
                    if (t > 0)
                        r = (t > 1 ? (t - 1) * Rn[n + 1][t - 2][u][v] : 0.0) + X * Rn[n + 1][t - 1][u][v];
                    else if (u > 0)
                        r = (u > 1 ? (u - 1) * Rn[n + 1][t][u - 2][v] : 0.0) + Y * Rn[n + 1][t][u - 1][v];
                    else
                        r = (v > 1 ? (v - 1) * Rn[n + 1][t][u][v - 2] : 0.0) + Z * Rn[n + 1][t][u][v - 1];
                    Rn[n][t][u][v] = r;
                }
    }
    for (int t = 0; t <= L; t++)
        for (int u = 0; u + t <= L; u++)
            for (int v = 0; v + u + t <= L; v++) R[t][u][v] = Rn[0][t][u][v];
}

/* ------------------------------------------------------------- Basis -- */
static void cart_powers(int l, int pw[OR_MAXCOMP][3])
{
    int c = 0;
    /* order: s; x y z; xx xy xz yy yz zz */
    for (int a = l; a >= 0; a--)
        for (int b = l - a; b >= 0; b--) {
            pw[c][0] = a;
            pw[c][1] = b;
            pw[c][2] = l - a - b;
            c++;
        }
}

static double dfact(int n) /* (n)!! with (-1)!! = 1 */
{
    double r = 1.0;
    for (int k = n; k > 1; k -= 2) r *= k;
    return r;
}

/* Overlap of two unnormalised primitive Cartesian Gaussians. */
static double prim_overlap(const int* pa, double a, const double* A, const int* pb, double b, const double* B)
{
    double s = pow(OR_PI / (a + b), 1.5);
    for (int x = 0; x < 3; x++) {
        etab E;
        hermite_E(pa[x], pb[x], a, b, A[x], B[x], E);
        s *= E[pa[x]][pb[x]][0];
    }
    return s;
}

void* or_create(int n_atoms, const int* Z, const double* xyz, int n_shells, const int* atom, const int* l,
                const int* nprim, const double* exps, const double* coefs)
{
    or_ctx* c = (or_ctx*)calloc(1, sizeof(or_ctx));
    c->n_atoms = n_atoms;
    c->n_shells = n_shells;
    c->Z = (double*)malloc(sizeof(double) * n_atoms);
    c->xyz = (double*)malloc(sizeof(double) * 3 * n_atoms);
    for (int a = 0; a < n_atoms; a++) {
        c->Z[a] = Z[a];
        for (int x = 0; x < 3; x++) c->xyz[3 * a + x] = xyz[3 * a + x];
    }
    c->sh = (or_shell*)calloc(n_shells, sizeof(or_shell));
    int off = 0, bf = 0;
    for (int s = 0; s < n_shells; s++) {
        or_shell* S = &c->sh[s];
        if (l[s] < 0 || l[s] > OR_MAXL || nprim[s] < 1 || nprim[s] > OR_MAXPRIM) {
            free(c->sh); free(c->Z); free(c->xyz); free(c);
            return NULL;
        }
        S->l = l[s];
        S->nprim = nprim[s];
        S->ncomp = (l[s] + 1) * (l[s] + 2) / 2;
        S->bf0 = bf;
        S->atom = atom[s];
        for (int x = 0; x < 3; x++) S->A[x] = xyz[3 * atom[s] + x];
        cart_powers(S->l, S->pw);
        for (int k = 0; k < S->nprim; k++) S->alpha[k] = exps[off + k];
        for (int m = 0; m < S->ncomp; m++) {
            const int* pw = S->pw[m];
            /* normalised primitive: (2a/pi)^{3/4} (4a)^{l/2} / sqrt((2i-1)!!(2j-1)!!(2k-1)!!) */
            double raw[OR_MAXPRIM];
            for (int k = 0; k < S->nprim; k++) {
                double a = S->alpha[k];
                raw[k] = coefs[off + k] * pow(2.0 * a / OR_PI, 0.75) * pow(4.0 * a, 0.5 * S->l)
                       / sqrt(dfact(2 * pw[0] - 1) * dfact(2 * pw[1] - 1) * dfact(2 * pw[2] - 1));
            }
            /* rescale the contracted component so that its self-overlap is exactly 1 */
            double ss = 0.0;
            for (int k = 0; k < S->nprim; k++)
                for (int q = 0; q < S->nprim; q++)
                    ss += raw[k] * raw[q] * prim_overlap(pw, S->alpha[k], S->A, pw, S->alpha[q], S->A);
            for (int k = 0; k < S->nprim; k++) S->d[m][k] = raw[k] / sqrt(ss);
        }
        off += nprim[s];
        bf += S->ncomp;
    }
    c->n_bf = bf;
    return c;
}

void or_destroy(void* h)
{
    or_ctx* c = (or_ctx*)h;
    if (!c) return;
    free(c->sh);
    free(c->Z);
    free(c->xyz);
    free(c);
}

int or_nbf(void* h) { return ((or_ctx*)h)->n_bf; }

void or_shell_info(void* h, int* bf0, int* ncomp)
{
    or_ctx* c = (or_ctx*)h;
    for (int s = 0; s < c->n_shells; s++) {
        bf0[s] = c->sh[s].bf0;
        ncomp[s] = c->sh[s].ncomp;
    }
}

/* ------------------------------------------------- One-electron terms -- */
double or_nuclear_repulsion(void* h)
{
    or_ctx* c = (or_ctx*)h;
    double e = 0.0;
    for (int a = 0; a < c->n_atoms; a++)
        for (int b = 0; b < a; b++) {
            double dx = c->xyz[3 * a] - c->xyz[3 * b], dy = c->xyz[3 * a + 1] - c->xyz[3 * b + 1],
                   dz = c->xyz[3 * a + 2] - c->xyz[3 * b + 2];
            e += c->Z[a] * c->Z[b] / sqrt(dx * dx + dy * dy + dz * dz);
        }
    return e;
}

/* S, T (kinetic) and V (nuclear attraction), N x N row-major. */
void or_one_electron(void* h, double* S, double* T, double* V)
{
    or_ctx* c = (or_ctx*)h;
    int N = c->n_bf;
    memset(S, 0, sizeof(double) * N * N);
    memset(T, 0, sizeof(double) * N * N);
    memset(V, 0, sizeof(double) * N * N);
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < c->n_shells; i++) {
        const or_shell* A = &c->sh[i];
        for (int j = 0; j < c->n_shells; j++) {
            const or_shell* B = &c->sh[j];
            for (int ka = 0; ka < A->nprim; ka++)
                for (int kb = 0; kb < B->nprim; kb++) {
                    double a = A->alpha[ka], b = B->alpha[kb], p = a + b;
                    double P[3];
                    etab E[3];
                    for (int x = 0; x < 3; x++) {
                        P[x] = (a * A->A[x] + b * B->A[x]) / p;
                        hermite_E(A->l, B->l + 2, a, b, A->A[x], B->A[x], E[x]);
                    }
                    /* nuclear attraction Hermite integrals, one table per nucleus */
                    int L = A->l + B->l;
                    for (int ma = 0; ma < A->ncomp; ma++)
                        for (int mb = 0; mb < B->ncomp; mb++) {
                            const int* pa = A->pw[ma];
                            const int* pb = B->pw[mb];
                            double cc = A->d[ma][ka] * B->d[mb][kb];
                            double s1[3], t1[3];
                            for (int x = 0; x < 3; x++) {
                                double sq = sqrt(OR_PI / p);
                                int ii = pa[x], jj = pb[x];
                                s1[x] = E[x][ii][jj][0] * sq;
                                double sp2 = E[x][ii][jj + 2][0] * sq;
                                double sm2 = jj >= 2 ? E[x][ii][jj - 2][0] * sq : 0.0;
                                t1[x] = -2.0 * b * b * sp2 + b * (2 * jj + 1) * s1[x] - 0.5 * jj * (jj - 1) * sm2;
                            }
                            int row = A->bf0 + ma, col = B->bf0 + mb;
                            S[row * N + col] += cc * s1[0] * s1[1] * s1[2];
                            T[row * N + col] += cc * (t1[0] * s1[1] * s1[2] + s1[0] * t1[1] * s1[2]
                                                      + s1[0] * s1[1] * t1[2]);
                        }
                    for (int nuc = 0; nuc < c->n_atoms; nuc++) {
                        double R[RN][RN][RN];
                        const double* C = &c->xyz[3 * nuc];
                        hermite_R(L, p, P[0] - C[0], P[1] - C[1], P[2] - C[2], R);
                        double pref = -c->Z[nuc] * 2.0 * OR_PI / p;
                        for (int ma = 0; ma < A->ncomp; ma++)
                            for (int mb = 0; mb < B->ncomp; mb++) {
                                const int* pa = A->pw[ma];
                                const int* pb = B->pw[mb];
                                double acc = 0.0;
                                for (int t = 0; t <= pa[0] + pb[0]; t++)
                                    for (int u = 0; u <= pa[1] + pb[1]; u++)
                                        for (int v = 0; v <= pa[2] + pb[2]; v++)
                                            acc += E[0][pa[0]][pb[0]][t] * E[1][pa[1]][pb[1]][u]
                                                 * E[2][pa[2]][pb[2]][v] * R[t][u][v];
                                V[(A->bf0 + ma) * N + B->bf0 + mb] += A->d[ma][ka] * B->d[mb][kb] * pref * acc;
                            }
                    }
                }
        }
    }
}

/*
 * One unnormalised primitive pair: out[0] = overlap, out[1] = kinetic energy,
 * out[2] = attraction to a point charge Zc at C (negative for Zc > 0).
 */
void or_one_electron_primitive(const int* pa, double a, const double* A, const int* pb, double b, const double* B,
                               double Zc, const double* C, double* out)
{
    double p = a + b, P[3];
    etab E[3];
    for (int x = 0; x < 3; x++) {
        P[x] = (a * A[x] + b * B[x]) / p;
        hermite_E(pa[x], pb[x] + 2, a, b, A[x], B[x], E[x]);
    }
    double s1[3], t1[3], sq = sqrt(OR_PI / p);
    for (int x = 0; x < 3; x++) {
        int ii = pa[x], jj = pb[x];
        s1[x] = E[x][ii][jj][0] * sq;
        double sp2 = E[x][ii][jj + 2][0] * sq;
        double sm2 = jj >= 2 ? E[x][ii][jj - 2][0] * sq : 0.0;
        t1[x] = -2.0 * b * b * sp2 + b * (2 * jj + 1) * s1[x] - 0.5 * jj * (jj - 1) * sm2;
    }
    out[0] = s1[0] * s1[1] * s1[2];
    out[1] = t1[0] * s1[1] * s1[2] + s1[0] * t1[1] * s1[2] + s1[0] * s1[1] * t1[2];
    int L = pa[0] + pa[1] + pa[2] + pb[0] + pb[1] + pb[2];
    double R[RN][RN][RN];
    hermite_R(L, p, P[0] - C[0], P[1] - C[1], P[2] - C[2], R);
    double acc = 0.0;
    for (int t = 0; t <= pa[0] + pb[0]; t++)
        for (int u = 0; u <= pa[1] + pb[1]; u++)
            for (int v = 0; v <= pa[2] + pb[2]; v++) acc += E[0][pa[0]][pb[0]][t] * E[1][pa[1]][pb[1]][u] * E[2][pa[2]][pb[2]][v] * R[t][u][v];
    out[2] = -Zc * 2.0 * OR_PI / p * acc;
}

/* ------------------------------------------------------ Two-electron -- */
/*
 * Contracted shell-quartet block (ab|cd), out[((a*nb+b)*nc+c)*nd+d], by the
 * McMurchie-Davidson expansion
 *   (ab|cd) = 2 pi^{5/2} / (p q sqrt(p+q)) sum_{tuv} E^{ab}_{tuv}
 *             sum_{tau nu phi} (-1)^{tau+nu+phi} E^{cd}_{tau nu phi} R_{t+tau,u+nu,v+phi}(pq/(p+q), P-Q)
 * summed over all primitive quartets with the final contraction coefficients.
 */
static void eri_block(const or_shell* A, const or_shell* B, const or_shell* C, const or_shell* D, double* out)
{
    int na = A->ncomp, nb = B->ncomp, nc = C->ncomp, nd = D->ncomp;
    int L = A->l + B->l + C->l + D->l;
    int Lab = A->l + B->l;
    memset(out, 0, sizeof(double) * na * nb * nc * nd);
    /* W[cd][t][u][v] = sum_{tau nu phi} (-1)^{tau+nu+phi} E^{cd}... R_{t+tau,...} */
    static __thread double W[OR_MAXCOMP * OR_MAXCOMP][2 * OR_MAXL + 1][2 * OR_MAXL + 1][2 * OR_MAXL + 1];
    for (int ka = 0; ka < A->nprim; ka++)
        for (int kb = 0; kb < B->nprim; kb++) {
            double a = A->alpha[ka], b = B->alpha[kb], p = a + b;
            double P[3];
            etab Eab[3];
            for (int x = 0; x < 3; x++) {
                P[x] = (a * A->A[x] + b * B->A[x]) / p;
                hermite_E(A->l, B->l, a, b, A->A[x], B->A[x], Eab[x]);
            }
            for (int kc = 0; kc < C->nprim; kc++)
                for (int kd = 0; kd < D->nprim; kd++) {
                    double c = C->alpha[kc], d = D->alpha[kd], q = c + d;
                    double Q[3];
                    etab Ecd[3];
                    for (int x = 0; x < 3; x++) {
                        Q[x] = (c * C->A[x] + d * D->A[x]) / q;
                        hermite_E(C->l, D->l, c, d, C->A[x], D->A[x], Ecd[x]);
                    }
                    double alpha = p * q / (p + q);
                    double R[RN][RN][RN];
                    hermite_R(L, alpha, P[0] - Q[0], P[1] - Q[1], P[2] - Q[2], R);
                    double pref = 2.0 * pow(OR_PI, 2.5) / (p * q * sqrt(p + q));
                    for (int mc = 0; mc < nc; mc++)
                        for (int md = 0; md < nd; md++) {
                            const int* pc = C->pw[mc];
                            const int* pd = D->pw[md];
                            int cd = mc * nd + md;
                            for (int t = 0; t <= Lab; t++)
                                for (int u = 0; u + t <= Lab; u++)
                                    for (int v = 0; v + u + t <= Lab; v++) {
                                        double acc = 0.0;
                                        for (int tau = 0; tau <= pc[0] + pd[0]; tau++)
                                            for (int nu = 0; nu <= pc[1] + pd[1]; nu++)
                                                for (int phi = 0; phi <= pc[2] + pd[2]; phi++) {
                                                    double sgn = ((tau + nu + phi) & 1) ? -1.0 : 1.0;
                                                    acc += sgn * Ecd[0][pc[0]][pd[0]][tau] * Ecd[1][pc[1]][pd[1]][nu]
                                                         * Ecd[2][pc[2]][pd[2]][phi] * R[t + tau][u + nu][v + phi];
                                                }
                                        W[cd][t][u][v] = acc;
                                    }
                        }
                    for (int ma = 0; ma < na; ma++)
                        for (int mb = 0; mb < nb; mb++) {
                            const int* pa = A->pw[ma];
                            const int* pb = B->pw[mb];
                            double cab = A->d[ma][ka] * B->d[mb][kb] * pref;
                            for (int mc = 0; mc < nc; mc++)
                                for (int md = 0; md < nd; md++) {
                                    int cd = mc * nd + md;
                                    double acc = 0.0;
                                    for (int t = 0; t <= pa[0] + pb[0]; t++)
                                        for (int u = 0; u <= pa[1] + pb[1]; u++)
                                            for (int v = 0; v <= pa[2] + pb[2]; v++)
                                                acc += Eab[0][pa[0]][pb[0]][t] * Eab[1][pa[1]][pb[1]][u]
                                                     * Eab[2][pa[2]][pb[2]][v] * W[cd][t][u][v];
                                    out[((ma * nb + mb) * nc + mc) * nd + md] +=
                                        cab * C->d[mc][kc] * D->d[md][kd] * acc;
                                }
                        }
                }
        }
}

void or_eri_shell_quartet(void* h, int i, int j, int k, int l, double* out)
{
    or_ctx* c = (or_ctx*)h;
    eri_block(&c->sh[i], &c->sh[j], &c->sh[k], &c->sh[l], out);
}

/* One unnormalised primitive Cartesian ERI (for derivative-identity checks). */
double or_eri_primitive(const int* pa, double a, const double* A, const int* pb, double b, const double* B,
                        const int* pc, double cexp, const double* C, const int* pd, double d, const double* D)
{
    or_shell s[4];
    const int* pw[4] = {pa, pb, pc, pd};
    double ex[4] = {a, b, cexp, d};
    const double* ctr[4] = {A, B, C, D};
    for (int q = 0; q < 4; q++) {
        memset(&s[q], 0, sizeof(or_shell));
        s[q].l = pw[q][0] + pw[q][1] + pw[q][2];
        s[q].nprim = 1;
        s[q].ncomp = 1;
        s[q].alpha[0] = ex[q];
        s[q].d[0][0] = 1.0;
        for (int x = 0; x < 3; x++) {
            s[q].A[x] = ctr[q][x];
            s[q].pw[0][x] = pw[q][x];
        }
    }
    double out;
    eri_block(&s[0], &s[1], &s[2], &s[3], &out);
    return out;
}

/* Q[i*n_shells+j] = sqrt(max_{mu in i, nu in j} |(mu nu|mu nu)|). */
void or_schwarz(void* h, double* Q)
{
    or_ctx* c = (or_ctx*)h;
    int n = c->n_shells;
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < n; i++) {
        double blk[OR_MAXCOMP * OR_MAXCOMP * OR_MAXCOMP * OR_MAXCOMP];
        for (int j = 0; j <= i; j++) {
            const or_shell *A = &c->sh[i], *B = &c->sh[j];
            eri_block(A, B, A, B, blk);
            double m = 0.0;
            int na = A->ncomp, nb = B->ncomp;
            for (int a = 0; a < na; a++)
                for (int b = 0; b < nb; b++) {
                    double v = fabs(blk[((a * nb + b) * na + a) * nb + b]);
                    if (v > m) m = v;
                }
            Q[i * n + j] = Q[j * n + i] = sqrt(m);
        }
    }
}

static inline int64_t pidx(int64_t a, int64_t b) { return a >= b ? a * (a + 1) / 2 + b : b * (b + 1) / 2 + a; }

int64_t or_packed_size(void* h)
{
    int64_t N = ((or_ctx*)h)->n_bf;
    int64_t np = N * (N + 1) / 2;
    return np * (np + 1) / 2;
}

/* Every symmetry-unique (mu nu|lam sig), stored at pidx(pidx(mu,nu), pidx(lam,sig)). */
void or_eri_packed(void* h, double* out)
{
    or_ctx* c = (or_ctx*)h;
    int n = c->n_shells;
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < n; i++) {
        double blk[OR_MAXCOMP * OR_MAXCOMP * OR_MAXCOMP * OR_MAXCOMP];
        for (int j = 0; j <= i; j++)
            for (int k = 0; k <= i; k++) {
                int lmax = (k == i) ? j : k;
                for (int l = 0; l <= lmax; l++) {
                    const or_shell *A = &c->sh[i], *B = &c->sh[j], *C = &c->sh[k], *D = &c->sh[l];
                    eri_block(A, B, C, D, blk);
                    for (int a = 0; a < A->ncomp; a++)
                        for (int b = 0; b < B->ncomp; b++)
                            for (int cc = 0; cc < C->ncomp; cc++)
                                for (int d = 0; d < D->ncomp; d++) {
                                    int64_t mu = A->bf0 + a, nu = B->bf0 + b, la = C->bf0 + cc, si = D->bf0 + d;
                                    out[pidx(pidx(mu, nu), pidx(la, si))] =
                                        blk[((a * B->ncomp + b) * C->ncomp + cc) * D->ncomp + d];
                                }
                }
            }
    }
}

/* J and K by their literal definitions over all ordered index quadruples. */
void or_jk_literal(int N, const double* eri, const double* P, double* J, double* K)
{
#pragma omp parallel for schedule(static)
    for (int mu = 0; mu < N; mu++)
        for (int nu = 0; nu < N; nu++) {
            double j = 0.0, k = 0.0;
            for (int la = 0; la < N; la++)
                for (int si = 0; si < N; si++) {
                    j += P[la * N + si] * eri[pidx(pidx(mu, nu), pidx(la, si))];
                    k += P[la * N + si] * eri[pidx(pidx(mu, la), pidx(nu, si))];
                }
            J[mu * N + nu] = j;
            K[mu * N + nu] = k;
        }
}

/*
 * J and K from the symmetry-unique shell quartets of Algorithm 1, each
 * integral X = (mu nu|lam sig) applied to the six Fock elements of Eq. 1a-1f
 * with weight f = 1/((1+d_ij)(1+d_kl)(1+d_ij,kl)):
 *   Jt_mu,nu += 4 f X P_lam,sig    Jt_lam,sig += 4 f X P_mu,nu
 *   Kt_mu,lam += 2 f X P_nu,sig    Kt_nu,sig  += 2 f X P_mu,lam
 *   Kt_mu,sig += 2 f X P_nu,lam    Kt_nu,lam  += 2 f X P_mu,sig
 * then J = (Jt + Jt^T)/2, K = (Kt + Kt^T)/2.  The loop bound on l is the
 * canonical one (l <= j when k == i, else l <= k).  Quartets whose Schwarz
 * bound Q_ij Q_kl is strictly below tau are skipped (tau = 0: none).
 * Thread-private accumulators, summed at the end (the private-Fock pattern
 * of Algorithm 2).  Returns the number of shell quartets evaluated.
 */
/* Wall-clock seconds (OpenMP's timer when available). */
static double wall_seconds(void)
{
#ifdef _OPENMP
    return omp_get_wtime();
#else
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return ts.tv_sec + 1e-9 * ts.tv_nsec;
#endif
}

static int64_t jk_unique_impl(void* h, const double* P, double tau, const double* Qsh, int64_t stride,
                              int64_t offset, const int64_t* rows, int64_t n_rows, double* J, double* K,
                              double* busy);

int64_t or_jk_unique(void* h, const double* P, double tau, const double* Qsh, double* J, double* K)
{
    return jk_unique_impl(h, P, tau, Qsh, 1, 0, NULL, 0, J, K, NULL);
}

/*
 * The same digestion restricted to an explicit list of bra pairs ij (rows of
 * Algorithm 1's outer loop, in any order; used to time a random sample of
 * rows of a large system).  Returns the quartets evaluated; *busy (if not
 * NULL) receives the seconds the threads spent in the rows, summed over
 * threads, so that a sample too small to keep every thread busy still
 * measures the work of its rows.
 */
int64_t or_jk_unique_rows(void* h, const double* P, double tau, const double* Qsh, int64_t n_rows, const int64_t* rows,
                          double* J, double* K, double* busy)
{
    return jk_unique_impl(h, P, tau, Qsh, 1, 0, rows, n_rows, J, K, busy);
}

/*
 * The same digestion restricted to the bra pairs ij = offset, offset+stride,
 * ... (a representative sample of Algorithm 1's outer loop, used to time the
 * oracle on large systems).  *unscreened receives the number of (ij, kl)
 * combinations the sampled rows span before screening.
 */
int64_t or_jk_unique_sample(void* h, const double* P, double tau, const double* Qsh, int64_t stride, int64_t offset,
                            double* J, double* K, int64_t* unscreened)
{
    or_ctx* c = (or_ctx*)h;
    int64_t np = (int64_t)c->n_shells * (c->n_shells + 1) / 2, u = 0;
    for (int64_t ij = offset; ij < np; ij += stride) u += ij + 1;
    *unscreened = u;
    return jk_unique_impl(h, P, tau, Qsh, stride, offset, NULL, 0, J, K, NULL);
}

static int64_t jk_unique_impl(void* h, const double* P, double tau, const double* Qsh, int64_t stride,
                              int64_t offset, const int64_t* rows, int64_t n_rows, double* J, double* K,
                              double* busy)
{
    or_ctx* c = (or_ctx*)h;
    int n = c->n_shells, N = c->n_bf;
    double* Jt = (double*)calloc((size_t)N * N, sizeof(double));
    double* Kt = (double*)calloc((size_t)N * N, sizeof(double));
    int64_t count = 0;
    double busy_sum = 0.0;
#pragma omp parallel reduction(+ : count, busy_sum)
    {
        double* Jp = (double*)calloc((size_t)N * N, sizeof(double));
        double* Kp = (double*)calloc((size_t)N * N, sizeof(double));
        double blk[OR_MAXCOMP * OR_MAXCOMP * OR_MAXCOMP * OR_MAXCOMP];
        const int64_t n_iter = rows ? n_rows : ((int64_t)n * (n + 1) / 2 - offset + stride - 1) / stride;
#pragma omp for schedule(dynamic, 1)
        for (int64_t it = 0; it < n_iter; it++) {
            const int64_t ij = rows ? rows[it] : offset + it * stride;
            const double t_row = busy ? wall_seconds() : 0.0;
            int i = (int)((sqrt(8.0 * ij + 1.0) - 1.0) / 2.0);
            while ((int64_t)i * (i + 1) / 2 > ij) i--;
            while ((int64_t)(i + 1) * (i + 2) / 2 <= ij) i++;
            int j = (int)(ij - (int64_t)i * (i + 1) / 2);
            for (int k = 0; k <= i; k++) {
                int lmax = (k == i) ? j : k;
                for (int l = 0; l <= lmax; l++) {
                    if (tau > 0.0 && Qsh[i * n + j] * Qsh[k * n + l] < tau) continue;
                    const or_shell *A = &c->sh[i], *B = &c->sh[j], *C = &c->sh[k], *D = &c->sh[l];
                    eri_block(A, B, C, D, blk);
                    count++;
                    double f = 1.0;
                    if (i == j) f *= 0.5;
                    if (k == l) f *= 0.5;
                    if (i == k && j == l) f *= 0.5;
                    for (int a = 0; a < A->ncomp; a++)
                        for (int b = 0; b < B->ncomp; b++)
                            for (int cc = 0; cc < C->ncomp; cc++)
                                for (int d = 0; d < D->ncomp; d++) {
                                    int mu = A->bf0 + a, nu = B->bf0 + b, la = C->bf0 + cc, si = D->bf0 + d;
                                    double X = f * blk[((a * B->ncomp + b) * C->ncomp + cc) * D->ncomp + d];
                                    Jp[mu * N + nu] += 4.0 * X * P[la * N + si];
                                    Jp[la * N + si] += 4.0 * X * P[mu * N + nu];
                                    Kp[mu * N + la] += 2.0 * X * P[nu * N + si];
                                    Kp[nu * N + si] += 2.0 * X * P[mu * N + la];
                                    Kp[mu * N + si] += 2.0 * X * P[nu * N + la];
                                    Kp[nu * N + la] += 2.0 * X * P[mu * N + si];
                                }
                }
            }
            if (busy) busy_sum += wall_seconds() - t_row;
        }
#pragma omp critical
        {
            for (int64_t x = 0; x < (int64_t)N * N; x++) {
                Jt[x] += Jp[x];
                Kt[x] += Kp[x];
            }
        }
        free(Jp);
        free(Kp);
    }
    for (int mu = 0; mu < N; mu++)
        for (int nu = 0; nu < N; nu++) {
            J[mu * N + nu] = 0.5 * (Jt[mu * N + nu] + Jt[nu * N + mu]);
            K[mu * N + nu] = 0.5 * (Kt[mu * N + nu] + Kt[nu * N + mu]);
        }
    free(Jt);
    free(Kt);
    if (busy) *busy = busy_sum;
    return count;
}

/*
 * Selected elements J_mu,nu and K_mu,nu by definition, summing over every
 * ordered shell pair (lam, sig); pairs are skipped when tau > 0 and the
 * Schwarz bound of the integral's quartet is strictly below tau.
 */
void or_jk_elements(void* h, const double* P, double tau, const double* Qsh, int n_el, const int* mu_list,
                    const int* nu_list, double* J_el, double* K_el)
{
    or_ctx* c = (or_ctx*)h;
    int n = c->n_shells, N = c->n_bf;
    int* shell_of = (int*)malloc(sizeof(int) * N);
    for (int s = 0; s < n; s++)
        for (int m = 0; m < c->sh[s].ncomp; m++) shell_of[c->sh[s].bf0 + m] = s;
    for (int e = 0; e < n_el; e++) {
        int mu = mu_list[e], nu = nu_list[e];
        int I = shell_of[mu], Jsh = shell_of[nu];
        int a = mu - c->sh[I].bf0, b = nu - c->sh[Jsh].bf0;
        double jsum = 0.0, ksum = 0.0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : jsum, ksum)
        for (int64_t kl = 0; kl < (int64_t)n * n; kl++) {
            int k = (int)(kl / n), l = (int)(kl % n);
            const or_shell *A = &c->sh[I], *B = &c->sh[Jsh], *C = &c->sh[k], *D = &c->sh[l];
            double blk[OR_MAXCOMP * OR_MAXCOMP * OR_MAXCOMP * OR_MAXCOMP];
            /* Coulomb: (mu nu | lam sig), lam in k, sig in l */
            if (!(tau > 0.0 && Qsh[I * n + Jsh] * Qsh[k * n + l] < tau)) {
                eri_block(A, B, C, D, blk);
                for (int cc = 0; cc < C->ncomp; cc++)
                    for (int d = 0; d < D->ncomp; d++)
                        jsum += P[(C->bf0 + cc) * N + D->bf0 + d]
                              * blk[((a * B->ncomp + b) * C->ncomp + cc) * D->ncomp + d];
            }
            /* Exchange: (mu lam | nu sig), lam in k, sig in l */
            if (!(tau > 0.0 && Qsh[I * n + k] * Qsh[Jsh * n + l] < tau)) {
                eri_block(A, C, B, D, blk);
                for (int cc = 0; cc < C->ncomp; cc++)
                    for (int d = 0; d < D->ncomp; d++)
                        ksum += P[(C->bf0 + cc) * N + D->bf0 + d]
                              * blk[((a * C->ncomp + cc) * B->ncomp + b) * D->ncomp + d];
            }
        }
        J_el[e] = jsum;
        K_el[e] = ksum;
    }
    free(shell_of);
}

/*
 * Whole shell blocks of J and K by definition: for each requested shell pair
 * (I, J), every component pair (mu in I, nu in J) of
 *   J_mu,nu = sum_{lam, sig} P_lam,sig (mu nu | lam sig)
 *   K_mu,nu = sum_{lam, sig} P_lam,sig (mu lam | nu sig)
 * summed over every ordered shell pair (k, l).  With tau > 0 an integral is
 * left out when the Schwarz bound of its own quartet is strictly below tau:
 * Q_IJ Q_kl for the Coulomb integrals, Q_Ik Q_Jl for the exchange ones.
 * Block b is written row-major (ncomp(I) x ncomp(J)) at offset off[b] of
 * J_out and K_out, off[b] = sum of the sizes of the blocks before it.
 */
void or_jk_shell_blocks(void* h, const double* P, double tau, const double* Qsh, int n_blk, const int* I_list,
                        const int* J_list, double* J_out, double* K_out)
{
    or_ctx* c = (or_ctx*)h;
    int n = c->n_shells, N = c->n_bf;
    int64_t off = 0;
    for (int e = 0; e < n_blk; e++) {
        const int I = I_list[e], Jsh = J_list[e];
        const or_shell *A = &c->sh[I], *B = &c->sh[Jsh];
        const int na = A->ncomp, nb = B->ncomp;
        double jacc[OR_MAXCOMP * OR_MAXCOMP] = {0}, kacc[OR_MAXCOMP * OR_MAXCOMP] = {0};
#pragma omp parallel
        {
            double jl[OR_MAXCOMP * OR_MAXCOMP] = {0}, kl_[OR_MAXCOMP * OR_MAXCOMP] = {0};
            double blk[OR_MAXCOMP * OR_MAXCOMP * OR_MAXCOMP * OR_MAXCOMP];
#pragma omp for schedule(dynamic, 4)
            for (int64_t kl = 0; kl < (int64_t)n * n; kl++) {
                const int k = (int)(kl / n), l = (int)(kl % n);
                const or_shell *C = &c->sh[k], *D = &c->sh[l];
                if (!(tau > 0.0 && Qsh[I * n + Jsh] * Qsh[k * n + l] < tau)) {
                    eri_block(A, B, C, D, blk); /* (a b | cc d) */
                    for (int a = 0; a < na; a++)
                        for (int b = 0; b < nb; b++) {
                            double s = 0.0;
                            for (int cc = 0; cc < C->ncomp; cc++)
                                for (int d = 0; d < D->ncomp; d++)
                                    s += P[(C->bf0 + cc) * N + D->bf0 + d]
                                       * blk[((a * nb + b) * C->ncomp + cc) * D->ncomp + d];
                            jl[a * nb + b] += s;
                        }
                }
                if (!(tau > 0.0 && Qsh[I * n + k] * Qsh[Jsh * n + l] < tau)) {
                    eri_block(A, C, B, D, blk); /* (a cc | b d) */
                    for (int a = 0; a < na; a++)
                        for (int b = 0; b < nb; b++) {
                            double s = 0.0;
                            for (int cc = 0; cc < C->ncomp; cc++)
                                for (int d = 0; d < D->ncomp; d++)
                                    s += P[(C->bf0 + cc) * N + D->bf0 + d]
                                       * blk[((a * C->ncomp + cc) * nb + b) * D->ncomp + d];
                            kl_[a * nb + b] += s;
                        }
                }
            }
#pragma omp critical
            for (int t = 0; t < na * nb; t++) {
                jacc[t] += jl[t];
                kacc[t] += kl_[t];
            }
        }
        for (int t = 0; t < na * nb; t++) {
            J_out[off + t] = jacc[t];
            K_out[off + t] = kacc[t];
        }
        off += na * nb;
    }
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
