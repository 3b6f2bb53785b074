/*
 * CPU oracle for the distance-preconditioned O(a)-improved Wilson-clover
 * operator -- TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark may load this code; the product path
 * never calls it.
 *
 * Plain FP64 C on the full lattice (no even-odd split), lexicographic sites,
 * explicit 4x4 gamma matrices (no spin projection), uncompressed 3x3 links.
 * It shares no source with the GPU library.
 *
 * Conventions: dims = {T, Lx, Ly, Lz}; coordinate c = {t, x, y, z};
 * site i = ((t*Lz + z)*Ly + y)*Lx + x.  Links U[i][mu][a][b] (row a, col b),
 * spinors psi[rhs][i][spin][colour], all double complex.
 *
 * Operator (Sec. II: O(a)-improved Wilson operator; modified covariant
 * derivatives of Sec. II for the time direction and eq. (redefcovs) of
 * Sec. III for all four directions):
 *
 *   (D'+M) psi(x) = (4+M) psi(x)
 *        - 1/2 sum_mu [ f_mu(x_mu) (1-gamma_mu) U_mu(x) psi(x+mu)
 *                     + b_mu(x_mu) (1+gamma_mu) U_mu(x-mu)^dag psi(x-mu) ]
 *        + c_sw (i/4) sum_{mu,nu} sigma_{mu nu} Fhat_{mu nu}(x) psi(x)
 *
 * The hop coefficients f, b are supplied by the caller per direction and
 * coordinate (they carry the profile ratios and the boundary sign).
 * Fhat_{mu nu} = (Q_{mu nu} - Q_{mu nu}^dag)/8 with Q the sum of the four
 * plaquette leaves at x in the (mu, nu) plane.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static void coords_of(const int d[4], long i, int c[4])
{
    c[1] = (int)(i % d[1]); i /= d[1];
    c[2] = (int)(i % d[2]); i /= d[2];
    c[3] = (int)(i % d[3]); i /= d[3];
    c[0] = (int)i;
}

static long index_of(const int d[4], const int c[4])
{
    return (((long)c[0] * d[3] + c[3]) * d[2] + c[2]) * d[1] + c[1];
}

/* neighbour of site i displaced by s (=+1 or -1) along mu, periodic wrap */
static long shift(const int d[4], long i, int mu, int s)
{
    int c[4];
    coords_of(d, i, c);
    c[mu] = (c[mu] + s + d[mu]) % d[mu];
    return index_of(d, c);
}

static long volume(const int d[4]) { return (long)d[0] * d[1] * d[2] * d[3]; }

static const cplx *link(const cplx *U, long i, int mu) { return U + (i * 4 + mu) * 9; }

/* C = A B for 3x3 */
static void mm(const cplx *A, const cplx *B, cplx *C)
{
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            cplx s = 0;
            for (int k = 0; k < 3; k++) s += A[a * 3 + k] * B[k * 3 + b];
            C[a * 3 + b] = s;
        }
}

/* B = A^dag */
static void dag(const cplx *A, cplx *B)
{
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) B[a * 3 + b] = conj(A[b * 3 + a]);
}

/* product of four 3x3 matrices */
static void mm4(const cplx *A, const cplx *B, const cplx *C, const cplx *D, cplx *out)
{
    cplx t1[9], t2[9];
    mm(A, B, t1);
    mm(t1, C, t2);
    mm(t2, D, out);
}

/*
 * Hopping part, per RHS:
 * out(x) = -1/2 sum_mu [ fwd[mu][x_mu] (1-g_mu) U_mu(x) psi(x+mu)
 *                      + bwd[mu][x_mu] (1+g_mu) U_mu(x-mu)^dag psi(x-mu) ]
 * gam: [4][4][4] (mu, row, col); fwd/bwd: [4][ldt].
 */
void or_hop(const int *d, const cplx *U, const cplx *gam, const double *fwd,
            const double *bwd, int ldt, const cplx *psi, cplx *out, int nrhs)
{
    long V = volume(d);
    for (int r = 0; r < nrhs; r++) {
        const cplx *in = psi + (long)r * V * 12;
        cplx *o = out + (long)r * V * 12;
#pragma omp parallel for schedule(static)
        for (long i = 0; i < V; i++) {
            int c[4];
            coords_of(d, i, c);
            cplx acc[12];
            for (int k = 0; k < 12; k++) acc[k] = 0;
            for (int mu = 0; mu < 4; mu++) {
                const cplx *g = gam + mu * 16;
                /* forward: (1 - gamma_mu) U_mu(x) psi(x+mu) */
                long jp = shift(d, i, mu, +1);
                const cplx *Uf = link(U, i, mu);
                cplx v[12], w[12];
                for (int s = 0; s < 4; s++)
                    for (int a = 0; a < 3; a++) {
                        cplx t = 0;
                        for (int b = 0; b < 3; b++) t += Uf[a * 3 + b] * in[jp * 12 + s * 3 + b];
                        v[s * 3 + a] = t;
                    }
                for (int s = 0; s < 4; s++)
                    for (int a = 0; a < 3; a++) {
                        cplx t = v[s * 3 + a];
                        for (int sp = 0; sp < 4; sp++) t -= g[s * 4 + sp] * v[sp * 3 + a];
                        w[s * 3 + a] = t;
                    }
                double cf = fwd[mu * ldt + c[mu]];
                for (int k = 0; k < 12; k++) acc[k] += cf * w[k];
                /* backward: (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu) */
                long jm = shift(d, i, mu, -1);
                const cplx *Ub = link(U, jm, mu);
                for (int s = 0; s < 4; s++)
                    for (int a = 0; a < 3; a++) {
                        cplx t = 0;
                        for (int b = 0; b < 3; b++) t += conj(Ub[b * 3 + a]) * in[jm * 12 + s * 3 + b];
                        v[s * 3 + a] = t;
                    }
                for (int s = 0; s < 4; s++)
                    for (int a = 0; a < 3; a++) {
                        cplx t = v[s * 3 + a];
                        for (int sp = 0; sp < 4; sp++) t += g[s * 4 + sp] * v[sp * 3 + a];
                        w[s * 3 + a] = t;
                    }
                double cb = bwd[mu * ldt + c[mu]];
                for (int k = 0; k < 12; k++) acc[k] += cb * w[k];
            }
            for (int k = 0; k < 12; k++) o[i * 12 + k] = -0.5 * acc[k];
        }
    }
}

/*
 * Field strength Fhat_{mu nu}(x) for all ordered pairs (mu, nu), mu != nu,
 * F[i][mu][nu][3][3]; the diagonal mu == nu is set to zero.
 * Q_{mu nu}(x) = sum of the four counter-clockwise plaquette leaves at x.
 */
void or_field_strength(const int *d, const cplx *U, cplx *F)
{
    long V = volume(d);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < V; i++) {
        for (int mu = 0; mu < 4; mu++)
            for (int nu = 0; nu < 4; nu++) {
                cplx *f = F + ((i * 4 + mu) * 4 + nu) * 9;
                if (mu == nu) {
                    for (int k = 0; k < 9; k++) f[k] = 0;
                    continue;
                }
                long xpm = shift(d, i, mu, +1), xpn = shift(d, i, nu, +1);
                long xmm = shift(d, i, mu, -1), xmn = shift(d, i, nu, -1);
                long xmm_pn = shift(d, xmm, nu, +1);
                long xmm_mn = shift(d, xmm, nu, -1);
                long xmn_pm = shift(d, xmn, mu, +1);
                cplx a[9], b[9], c[9], e[9], leaf[9], Q[9];
                for (int k = 0; k < 9; k++) Q[k] = 0;
                /* leaf 1: x -> x+mu -> x+mu+nu -> x+nu -> x */
                dag(link(U, xpn, mu), a);
                dag(link(U, i, nu), b);
                mm4(link(U, i, mu), link(U, xpm, nu), a, b, leaf);
                for (int k = 0; k < 9; k++) Q[k] += leaf[k];
                /* leaf 2: x -> x+nu -> x+nu-mu -> x-mu -> x */
                dag(link(U, xmm_pn, mu), a);
                dag(link(U, xmm, nu), b);
                mm4(link(U, i, nu), a, b, link(U, xmm, mu), leaf);
                for (int k = 0; k < 9; k++) Q[k] += leaf[k];
                /* leaf 3: x -> x-mu -> x-mu-nu -> x-nu -> x */
                dag(link(U, xmm, mu), a);
                dag(link(U, xmm_mn, nu), b);
                mm4(a, b, link(U, xmm_mn, mu), link(U, xmn, nu), leaf);
                for (int k = 0; k < 9; k++) Q[k] += leaf[k];
                /* leaf 4: x -> x-nu -> x-nu+mu -> x+mu -> x */
                dag(link(U, xmn, nu), c);
                dag(link(U, i, mu), e);
                mm4(c, link(U, xmn, mu), link(U, xmn_pm, nu), e, leaf);
                for (int k = 0; k < 9; k++) Q[k] += leaf[k];
                for (int p = 0; p < 3; p++)
                    for (int q = 0; q < 3; q++)
                        f[p * 3 + q] = (Q[p * 3 + q] - conj(Q[q * 3 + p])) / 8.0;
            }
    }
}

/*
 * Clover term: out(x) = c_sw (i/4) sum_{mu,nu} sigma_{mu nu} Fhat_{mu nu}(x) psi(x)
 * sigma: [4][4][4][4] (mu, nu, row, col).
 */
void or_clover(const int *d, const cplx *F, const cplx *sigma, double csw,
               const cplx *psi, cplx *out, int nrhs)
{
    long V = volume(d);
    for (int r = 0; r < nrhs; r++) {
        const cplx *in = psi + (long)r * V * 12;
        cplx *o = out + (long)r * V * 12;
#pragma omp parallel for schedule(static)
        for (long i = 0; i < V; i++) {
            cplx acc[12];
            for (int k = 0; k < 12; k++) acc[k] = 0;
            for (int mu = 0; mu < 4; mu++)
                for (int nu = 0; nu < 4; nu++) {
                    if (mu == nu) continue;
                    const cplx *f = F + ((i * 4 + mu) * 4 + nu) * 9;
                    const cplx *sg = sigma + (mu * 4 + nu) * 16;
                    for (int s = 0; s < 4; s++)
                        for (int a = 0; a < 3; a++) {
                            cplx t = 0;
                            for (int sp = 0; sp < 4; sp++)
                                for (int b = 0; b < 3; b++)
                                    t += sg[s * 4 + sp] * f[a * 3 + b] * in[i * 12 + sp * 3 + b];
                            acc[s * 3 + a] += t;
                        }
                }
            for (int k = 0; k < 12; k++) o[i * 12 + k] = csw * 0.25 * I * acc[k];
        }
    }
}

/*
 * The same clover term as a 12x12 matrix per site, Cm[i][row][col] with
 * row/col = spin*3 + colour: Cm = c_sw (i/4) sum_{mu,nu} sigma_{mu nu} (x) Fhat_{mu nu}.
 */
void or_clover_matrix(const int *d, const cplx *F, const cplx *sigma, double csw, cplx *Cm)
{
    long V = volume(d);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < V; i++) {
        cplx *m = Cm + i * 144;
        for (int k = 0; k < 144; k++) m[k] = 0;
        for (int mu = 0; mu < 4; mu++)
            for (int nu = 0; nu < 4; nu++) {
                if (mu == nu) continue;
                const cplx *f = F + ((i * 4 + mu) * 4 + nu) * 9;
                const cplx *sg = sigma + (mu * 4 + nu) * 16;
                for (int s = 0; s < 4; s++)
                    for (int a = 0; a < 3; a++)
                        for (int sp = 0; sp < 4; sp++)
                            for (int b = 0; b < 3; b++)
                                m[(s * 3 + a) * 12 + sp * 3 + b] += csw * 0.25 * I * sg[s * 4 + sp] * f[a * 3 + b];
            }
    }
}

/* out(x) = Cm(x) psi(x) */
static void clover_mat_apply(const int *d, const cplx *Cm, const cplx *psi, cplx *out, int nrhs)
{
    long V = volume(d);
    for (int r = 0; r < nrhs; r++) {
        const cplx *in = psi + (long)r * V * 12;
        cplx *o = out + (long)r * V * 12;
#pragma omp parallel for schedule(static)
        for (long i = 0; i < V; i++) {
            const cplx *m = Cm + i * 144;
            for (int k = 0; k < 12; k++) {
                cplx t = 0;
                for (int l = 0; l < 12; l++) t += m[k * 12 + l] * in[i * 12 + l];
                o[i * 12 + k] = t;
            }
        }
    }
}

/* full operator: out = (4+M) psi + hop(psi) + clover(psi); Cm NULL: no clover */
void or_dirac(const int *d, const cplx *U, const cplx *Cm, const cplx *gam, double M,
              const double *fwd, const double *bwd, int ldt, const cplx *psi, cplx *out,
              int nrhs)
{
    long n = volume(d) * 12 * (long)nrhs;
    or_hop(d, U, gam, fwd, bwd, ldt, psi, out, nrhs);
    if (Cm) {
        cplx *tmp = (cplx *)malloc(sizeof(cplx) * n);
        clover_mat_apply(d, Cm, psi, tmp, nrhs);
#pragma omp parallel for schedule(static)
        for (long k = 0; k < n; k++) out[k] += tmp[k];
        free(tmp);
    }
#pragma omp parallel for schedule(static)
    for (long k = 0; k < n; k++) out[k] += (4.0 + M) * psi[k];
}

static cplx dot(const cplx *a, const cplx *b, long n)
{
    double re = 0, im = 0;
#pragma omp parallel for reduction(+ : re, im) schedule(static)
    for (long k = 0; k < n; k++) {
        cplx t = conj(a[k]) * b[k];
        re += creal(t);
        im += cimag(t);
    }
    return re + I * im;
}

static double norm2(const cplx *a, long n) { return creal(dot(a, a, n)); }

/*
 * BiCGStab (van der Vorst) on the full lattice, one RHS at a time.
 * Stops when |b - A x|_2 / |b|_2 < tol, measured on the recomputed true
 * residual; on a recursive-residual stop that the true residual does not
 * confirm, or on a breakdown (rho or omega vanishing), it restarts from the
 * true residual.  x holds the initial guess on entry and the solution on exit.
 * iters[r] receives the number of operator applications pairs, relres[r] the
 * final true relative residual.  Returns 0 if every RHS converged, else 1.
 */
int or_bicgstab(const int *d, const cplx *U, const cplx *Cm, const cplx *gam,
                double M, const double *fwd,
                const double *bwd, int ldt, const cplx *b_all, cplx *x_all,
                int nrhs, double tol, int maxit, int *iters, double *relres)
{
    long n = volume(d) * 12;
    cplx *r = malloc(sizeof(cplx) * n), *rh = malloc(sizeof(cplx) * n);
    cplx *p = malloc(sizeof(cplx) * n), *v = malloc(sizeof(cplx) * n);
    cplx *s = malloc(sizeof(cplx) * n), *t = malloc(sizeof(cplx) * n);
    int status = 0;
    for (int rr = 0; rr < nrhs; rr++) {
        const cplx *b = b_all + rr * n;
        cplx *x = x_all + rr * n;
        double bn = sqrt(norm2(b, n));
        int it = 0, done = 0;
        double rel = 0;
        if (bn == 0) {
            memset(x, 0, sizeof(cplx) * n);
            iters[rr] = 0;
            relres[rr] = 0;
            continue;
        }
        while (!done && it < maxit) {
            /* (re)start from the true residual */
            or_dirac(d, U, Cm, gam, M, fwd, bwd, ldt, x, r, 1);
            for (long k = 0; k < n; k++) r[k] = b[k] - r[k];
            rel = sqrt(norm2(r, n)) / bn;
            if (rel < tol) { done = 1; break; }
            memcpy(rh, r, sizeof(cplx) * n);
            memset(p, 0, sizeof(cplx) * n);
            memset(v, 0, sizeof(cplx) * n);
            cplx rho = 1, alpha = 1, omega = 1;
            while (it < maxit) {
                cplx rho_new = dot(rh, r, n);
                if (cabs(rho_new) == 0.0) break; /* breakdown: restart */
                cplx beta = (rho_new / rho) * (alpha / omega);
                for (long k = 0; k < n; k++) p[k] = r[k] + beta * (p[k] - omega * v[k]);
                or_dirac(d, U, Cm, gam, M, fwd, bwd, ldt, p, v, 1);
                cplx rv = dot(rh, v, n);
                if (cabs(rv) == 0.0) break;
                alpha = rho_new / rv;
                for (long k = 0; k < n; k++) s[k] = r[k] - alpha * v[k];
                or_dirac(d, U, Cm, gam, M, fwd, bwd, ldt, s, t, 1);
                it++;
                double tt = norm2(t, n);
                if (tt == 0.0) {
                    for (long k = 0; k < n; k++) x[k] += alpha * p[k];
                    break;
                }
                omega = dot(t, s, n) / tt;
                for (long k = 0; k < n; k++) {
                    x[k] += alpha * p[k] + omega * s[k];
                    r[k] = s[k] - omega * t[k];
                }
                rho = rho_new;
                if (sqrt(norm2(r, n)) / bn < tol) break;
                if (cabs(omega) == 0.0) break;
            }
            /* confirm on the true residual (next loop pass recomputes it) */
            or_dirac(d, U, Cm, gam, M, fwd, bwd, ldt, x, r, 1);
            for (long k = 0; k < n; k++) r[k] = b[k] - r[k];
            rel = sqrt(norm2(r, n)) / bn;
            if (rel < tol) done = 1;
        }
        iters[rr] = it;
        relres[rr] = rel;
        if (!done) status = 1;
    }
    free(r); free(rh); free(p); free(v); free(s); free(t);
    return status;
}

#ifdef _OPENMP
#include <omp.h>
#endif
/* number of host threads the oracle's parallel loops use */
int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
