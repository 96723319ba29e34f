/*
 * hisq_oracle.c -- plain, slow, obviously-correct FP64 CPU reference for the HISQ
 * staggered Dslash, the even-odd normal operator and the Krylov solvers built on it.
 *
 * TEST INFRASTRUCTURE ONLY.  It is loaded by the test suite, the smoke check and the
 * benchmark's CPU-baseline leg, never by the GPU library, and it shares no code,
 * header or table with that library.
 *
 * Conventions (all from the paper unless stated):
 *   - sites (x,y,z,t), mu = 0,1,2,3 = x,y,z,t (Sec. 3).
 *   - memory index of a site: floor(lex/2) + (V/2) * ((x+y+z+t) mod 2),
 *     lex = x + Nx (y + Ny (z + Nz t)); links at index + mu*V (Sec. 4.3 equations).
 *     (The paper writes N_sigma for Nx = Ny = Nz; the formula is used with the
 *     three spatial extents separately, which reduces to it when they are equal.)
 *   - links and spinors are row-major complex 3x3 / 3-vectors stored as
 *     interleaved (re, im) doubles.
 *   - Dslash (Sec. 5.1, Eq. for the stencil):
 *       (D phi)(x) = sum_{mu=0..3} eta_mu(x) [ X_mu(x) phi(x+mu) - X_mu(x-mu)^+ phi(x-mu)
 *                                         + W_mu(x) phi(x+3mu) - W_mu(x-3mu)^+ phi(x-3mu) ]
 *     The paper's sum "mu=0 to 4" is read as mu = 0..3 and its Naik link written at
 *     x+3mu is read as W_mu(x); the paper drops the staggered phases, which are taken
 *     here in the MILC convention eta_0 = 1, eta_1 = (-1)^x, eta_2 = (-1)^(x+y),
 *     eta_3 = (-1)^(x+y+z).  Spinors are periodic in space and antiperiodic in time
 *     (Sec. 3): every hop that wraps around t picks up a factor -1.  Links are
 *     periodic.  With `phased` = 1 the links are taken to contain eta and the time
 *     boundary sign already, and neither is applied.
 *   - M = 2m + D; on even sites A = M^+ M = 4m^2 - D_eo D_oe (D anti-Hermitian).
 *   - CG / multi-shift CG / flexible CG as described at each function.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

typedef struct {
    int n[4];
    long V, Vh;
} lattice;

static lattice make_lattice(const int dims[4])
{
    lattice L;
    for (int i = 0; i < 4; i++) L.n[i] = dims[i];
    L.V = (long)dims[0] * dims[1] * dims[2] * dims[3];
    L.Vh = L.V / 2;
    return L;
}

/* ------------------------------------------------------------------ indexing (Sec. 4.3) */

static long lex_of(const lattice *L, const int x[4])
{
    return x[0] + (long)L->n[0] * (x[1] + (long)L->n[1] * (x[2] + (long)L->n[2] * x[3]));
}

static int parity_of(const int x[4]) { return (x[0] + x[1] + x[2] + x[3]) & 1; }

static long eo_index(const lattice *L, const int x[4])
{
    return lex_of(L, x) / 2 + L->Vh * parity_of(x);
}

/* coordinates of the site with canonical index `idx` (inverse of eo_index) */
static void coords_of(const lattice *L, long idx, int x[4])
{
    int par = idx >= L->Vh;
    long half = idx - par * L->Vh;
    /* lex is 2*half or 2*half+1; exactly one of them has parity `par` */
    for (int b = 0; b < 2; b++) {
        long lex = 2 * half + b;
        int c[4];
        c[0] = (int)(lex % L->n[0]);
        c[1] = (int)((lex / L->n[0]) % L->n[1]);
        c[2] = (int)((lex / ((long)L->n[0] * L->n[1])) % L->n[2]);
        c[3] = (int)(lex / ((long)L->n[0] * L->n[1] * L->n[2]));
        if (parity_of(c) == par) {
            memcpy(x, c, sizeof c);
            return;
        }
    }
}

/* y = x + k * mu^ with periodic wrap; returns the spinor boundary sign of that hop
 * (-1 when a t-hop wraps around the lattice, Sec. 3), +1 otherwise. */
static double hop(const lattice *L, const int x[4], int mu, int k, int y[4])
{
    memcpy(y, x, 4 * sizeof(int));
    int v = x[mu] + k, n = L->n[mu];
    int wrapped = (v < 0 || v >= n);
    y[mu] = ((v % n) + n) % n;
    return (mu == 3 && wrapped) ? -1.0 : 1.0;
}

/* MILC staggered phase eta_mu(x) */
static double eta(int mu, const int x[4])
{
    int s = 0;
    for (int nu = 0; nu < mu; nu++) s += x[nu];
    return (s & 1) ? -1.0 : 1.0;
}

/* ------------------------------------------------------------------ SU(3) algebra with counters */

/* optional operation counting, used once per test to pin the paper's accounting */
static long g_flops, g_link_words, g_spinor_words, g_out_words;
static int g_count;

static const cplx *link_at(const lattice *L, const cplx *links, int mu, const int x[4])
{
    if (g_count) g_link_words += 18;
    return links + ((long)mu * L->V + eo_index(L, x)) * 9;
}

/* out = U v; 9 complex multiplications + 6 complex additions = 66 flops */
static void matvec(const cplx *U, const cplx *v, cplx *out)
{
    for (int i = 0; i < 3; i++)
        out[i] = U[3 * i + 0] * v[0] + U[3 * i + 1] * v[1] + U[3 * i + 2] * v[2];
    if (g_count) g_flops += 9 * 6 + 6 * 2;
}

/* out = U^+ v */
static void matvec_dag(const cplx *U, const cplx *v, cplx *out)
{
    for (int i = 0; i < 3; i++)
        out[i] = conj(U[0 * 3 + i]) * v[0] + conj(U[1 * 3 + i]) * v[1] + conj(U[2 * 3 + i]) * v[2];
    if (g_count) g_flops += 9 * 6 + 6 * 2;
}

/* acc += s * v (a complex 3-vector addition: 6 flops; s = +-1 is a sign, not counted) */
static void vadd(cplx *acc, double s, const cplx *v)
{
    for (int i = 0; i < 3; i++) acc[i] += s * v[i];
    if (g_count) g_flops += 6;
}

/* spinor of parity-field `f` (half-lattice field of the parity of y) at site y */
static const cplx *spinor_at(const lattice *L, const cplx *f, const int y[4])
{
    if (g_count) g_spinor_words += 6;
    return f + (eo_index(L, y) - L->Vh * parity_of(y)) * 3;
}

/* ------------------------------------------------------------------ Dslash */

/* The four hops of direction mu at site x, summed with the signs of the stencil:
 *   X_mu(x) phi(x+mu) - X_mu(x-mu)^+ phi(x-mu) + W_mu(x) phi(x+3mu) - W_mu(x-3mu)^+ phi(x-3mu)
 * including the spinor boundary signs of each hop (unless `phased`). */
static void direction_sum(const lattice *L, const cplx *fat, const cplx *lng, int phased,
                          const cplx *in, const int x[4], int mu, cplx out[3])
{
    int y[4];
    cplx t[3];
    double bc;

    bc = hop(L, x, mu, +1, y);
    matvec(link_at(L, fat, mu, x), spinor_at(L, in, y), out);
    if (!phased && bc < 0) for (int i = 0; i < 3; i++) out[i] = -out[i];

    bc = hop(L, x, mu, -1, y);
    matvec_dag(link_at(L, fat, mu, y), spinor_at(L, in, y), t);
    vadd(out, (phased ? 1.0 : bc) * -1.0, t);

    bc = hop(L, x, mu, +3, y);
    matvec(link_at(L, lng, mu, x), spinor_at(L, in, y), t);
    vadd(out, (phased ? 1.0 : bc), t);

    bc = hop(L, x, mu, -3, y);
    matvec_dag(link_at(L, lng, mu, y), spinor_at(L, in, y), t);
    vadd(out, (phased ? 1.0 : bc) * -1.0, t);
}

static void dslash_site(const lattice *L, const cplx *fat, const cplx *lng, int phased,
                        const cplx *in, const int x[4], cplx out[3])
{
    cplx d[3];
    for (int mu = 0; mu < 4; mu++) {
        direction_sum(L, fat, lng, phased, in, x, mu, d);
        double e = phased ? 1.0 : eta(mu, x);
        if (mu == 0) {
            for (int i = 0; i < 3; i++) out[i] = e * d[i];
        } else {
            vadd(out, e, d);
        }
    }
    if (g_count) g_out_words += 6;
}

/*
 * out = D_{p, 1-p} in: `in` holds the half-lattice field of parity 1-p, `out` receives the
 * half-lattice field of parity p = out_parity.  nrhs fields are stored one after another
 * ([nrhs][Vh][3] complex).
 */
void ho_dslash(const int dims[4], const double *fat, const double *lng, int phased,
               int out_parity, const double *in, double *out, int nrhs)
{
    lattice L = make_lattice(dims);
    const cplx *F = (const cplx *)fat, *W = (const cplx *)lng;
    for (int r = 0; r < nrhs; r++) {
        const cplx *src = (const cplx *)in + (long)r * L.Vh * 3;
        cplx *dst = (cplx *)out + (long)r * L.Vh * 3;
#pragma omp parallel for schedule(static)
        for (long s = 0; s < L.Vh; s++) {
            int x[4];
            coords_of(&L, s + out_parity * L.Vh, x);
            dslash_site(&L, F, W, phased, src, x, dst + s * 3);
        }
    }
}

/* Operation count of one output site: flops, link words, neighbour words, output words. */
void ho_count_site(const int dims[4], const double *fat, const double *lng, const double *in,
                   long out_index, long counts[4])
{
    lattice L = make_lattice(dims);
    int x[4];
    cplx out[3];
    coords_of(&L, out_index, x);
    g_flops = g_link_words = g_spinor_words = g_out_words = 0;
    g_count = 1;
    dslash_site(&L, (const cplx *)fat, (const cplx *)lng, 0, (const cplx *)in, x, out);
    g_count = 0;
    counts[0] = g_flops;
    counts[1] = g_link_words;
    counts[2] = g_spinor_words;
    counts[3] = g_out_words;
}

/* One output site of D (for sampled checks of very large lattices). */
void ho_dslash_site(const int dims[4], const double *fat, const double *lng, int phased,
                    const double *in, long out_index, double *out6)
{
    lattice L = make_lattice(dims);
    int x[4];
    coords_of(&L, out_index, x);
    dslash_site(&L, (const cplx *)fat, (const cplx *)lng, phased, (const cplx *)in, x, (cplx *)out6);
}

/* Fold eta_mu(x) and the time boundary sign into links: the result used with
 * phased = 1 reproduces the unphased operator.  naik_hops = 1 for X, 3 for W: the
 * link at x carries -1 when the hop x -> x + k t^ wraps. */
void ho_phase_links(const int dims[4], const double *links, double *out, int naik_hops)
{
    lattice L = make_lattice(dims);
    for (int mu = 0; mu < 4; mu++) {
#pragma omp parallel for schedule(static)
        for (long i = 0; i < L.V; i++) {
            int x[4], y[4];
            coords_of(&L, i, x);
            double s = eta(mu, x) * hop(&L, x, mu, naik_hops, y);
            const cplx *src = (const cplx *)links + ((long)mu * L.V + i) * 9;
            cplx *dst = (cplx *)out + ((long)mu * L.V + i) * 9;
            for (int k = 0; k < 9; k++) dst[k] = s * src[k];
        }
    }
}

void ho_eo_index(const int dims[4], const int x[4], long *idx)
{
    lattice L = make_lattice(dims);
    *idx = eo_index(&L, x);
}

void ho_coords(const int dims[4], long idx, int x[4])
{
    lattice L = make_lattice(dims);
    coords_of(&L, idx, x);
}

/* ------------------------------------------------------------------ vector algebra */

static cplx dot(const cplx *a, const cplx *b, long n) /* sum conj(a) b */
{
    double re = 0, im = 0;
#pragma omp parallel for reduction(+ : re, im) schedule(static)
    for (long i = 0; i < n; i++) {
        cplx p = conj(a[i]) * b[i];
        re += creal(p);
        im += cimag(p);
    }
    return re + I * im;
}

static double norm2(const cplx *a, long n) { return creal(dot(a, a, n)); }

/* ------------------------------------------------------------------ normal operator */

typedef struct {
    lattice L;
    const cplx *fat, *lng;
    int phased;
    double m;
    cplx *tmp; /* odd half-field */
} normal_op;

/* out = (4 m^2 - D_eo D_oe) in  on even sites (A = M^+ M with M = 2m + D) */
static void apply_A(normal_op *op, const cplx *in, cplx *out)
{
    const lattice *L = &op->L;
    ho_dslash(L->n, (const double *)op->fat, (const double *)op->lng, op->phased, 1,
              (const double *)in, (double *)op->tmp, 1);
    ho_dslash(L->n, (const double *)op->fat, (const double *)op->lng, op->phased, 0,
              (const double *)op->tmp, (double *)out, 1);
    double m4 = 4.0 * op->m * op->m;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < L->Vh * 3; i++) out[i] = m4 * in[i] - out[i];
}

void ho_mdagm(const int dims[4], const double *fat, const double *lng, int phased, double m,
              const double *in, double *out, int nrhs)
{
    normal_op op = {make_lattice(dims), (const cplx *)fat, (const cplx *)lng, phased, m, NULL};
    op.tmp = malloc(sizeof(cplx) * op.L.Vh * 3);
    for (int r = 0; r < nrhs; r++)
        apply_A(&op, (const cplx *)in + (long)r * op.L.Vh * 3, (cplx *)out + (long)r * op.L.Vh * 3);
    free(op.tmp);
}

/* ------------------------------------------------------------------ CG (Sec. 3.2) */

/*
 * Textbook conjugate gradient on A x = b (Hestenes-Stiefel), x0 taken from x.
 *   r = b - A x; p = r
 *   repeat: alpha = |r|^2 / <p, A p>;  x += alpha p;  r -= alpha A p;
 *           beta = |r_new|^2 / |r|^2;  p = r + beta p
 * until |r| <= tol |b| (iterated residual).  stats: [iterations, |r|/|b| iterated,
 * |b - A x|/|b| recomputed].  Returns 0 when the recomputed residual meets tol.
 */
int ho_cg(const int dims[4], const double *fat, const double *lng, int phased, double m,
          const double *bv, double *xv, double tol, int maxiter, double stats[3])
{
    normal_op op = {make_lattice(dims), (const cplx *)fat, (const cplx *)lng, phased, m, NULL};
    long n = op.L.Vh * 3;
    const cplx *b = (const cplx *)bv;
    cplx *x = (cplx *)xv;
    cplx *r = malloc(sizeof(cplx) * n), *p = malloc(sizeof(cplx) * n), *Ap = malloc(sizeof(cplx) * n);
    op.tmp = malloc(sizeof(cplx) * n);

    apply_A(&op, x, Ap);
    for (long i = 0; i < n; i++) r[i] = b[i] - Ap[i];
    memcpy(p, r, sizeof(cplx) * n);
    double bb = norm2(b, n), rr = norm2(r, n);
    int k = 0;
    while (k < maxiter && rr > tol * tol * bb) {
        apply_A(&op, p, Ap);
        double pAp = creal(dot(p, Ap, n));
        double alpha = rr / pAp;
#pragma omp parallel for schedule(static)
        for (long i = 0; i < n; i++) {
            x[i] += alpha * p[i];
            r[i] -= alpha * Ap[i];
        }
        double rr_new = norm2(r, n);
        double beta = rr_new / rr;
        rr = rr_new;
#pragma omp parallel for schedule(static)
        for (long i = 0; i < n; i++) p[i] = r[i] + beta * p[i];
        k++;
    }
    apply_A(&op, x, Ap);
    for (long i = 0; i < n; i++) r[i] = b[i] - Ap[i];
    stats[0] = k;
    stats[1] = sqrt(rr / bb);
    stats[2] = sqrt(norm2(r, n) / bb);
    free(r); free(p); free(Ap); free(op.tmp);
    return stats[2] <= tol ? 0 : 1;
}

/* A fixed number of CG iterations from x0 = 0 (used to time the oracle on a bounded sample). */
double ho_cg_fixed(const int dims[4], const double *fat, const double *lng, double m,
                   const double *bv, double *xv, int iters)
{
    double stats[3];
    memset(xv, 0, sizeof(cplx) * (size_t)make_lattice(dims).Vh * 3);
    ho_cg(dims, fat, lng, 0, m, bv, xv, 0.0, iters, stats);
    return stats[1];
}

/* ------------------------------------------------------------------ multi-shift CG */

/*
 * Multi-shift CG (shift-invariance of the Krylov space, Sec. 3.2 and its reference to
 * Jegerlehner): solves (A + sigma_s) x_s = b for all s, with one application of A + sigma_0
 * per iteration, sigma_0 = min sigma, delta_s = sigma_s - sigma_0.
 *   r = b, p_s = b, x_s = 0, zeta_s^{-1} = zeta_s^0 = 1, alpha_{-1} = 1, beta_{-1} = 0
 *   q = (A + sigma_0) p_0;  alpha = |r|^2 / <p_0, q>
 *   zeta_s^{n+1} = zeta_s^n zeta_s^{n-1} alpha_{n-1} /
 *        [alpha_{n-1} zeta_s^{n-1} (1 + alpha delta_s) + alpha beta_{n-1} (zeta_s^{n-1} - zeta_s^n)]
 *   alpha_s = alpha zeta_s^{n+1} / zeta_s^n;  x_s += alpha_s p_s
 *   r -= alpha q;  beta = |r_new|^2/|r|^2;  beta_s = beta (zeta_s^{n+1}/zeta_s^n)^2
 *   p_s = zeta_s^{n+1} r + beta_s p_s
 * Shift s is frozen once |zeta_s| |r| <= tol_s |b|.  x is [nshift][Vh][3].
 * stats: [iterations, then per shift the recomputed |b - (A+sigma_s) x_s| / |b|].
 */
int ho_multishift_cg(const int dims[4], const double *fat, const double *lng, int phased,
                     double m, int nshift, const double *sigma, const double *bv, double *xv,
                     const double *tol, int maxiter, double *stats)
{
    normal_op op = {make_lattice(dims), (const cplx *)fat, (const cplx *)lng, phased, m, NULL};
    long n = op.L.Vh * 3;
    const cplx *b = (const cplx *)bv;
    cplx *x = (cplx *)xv;
    int s0 = 0;
    for (int s = 1; s < nshift; s++)
        if (sigma[s] < sigma[s0]) s0 = s;
    cplx *r = malloc(sizeof(cplx) * n), *q = malloc(sizeof(cplx) * n);
    cplx *p = malloc(sizeof(cplx) * n * nshift);
    op.tmp = malloc(sizeof(cplx) * n);
    double *zeta = malloc(sizeof(double) * nshift), *zeta_old = malloc(sizeof(double) * nshift);
    int *active = malloc(sizeof(int) * nshift);
    for (int s = 0; s < nshift; s++) {
        zeta[s] = zeta_old[s] = 1.0;
        active[s] = 1;
        memcpy(p + (long)s * n, b, sizeof(cplx) * n);
        memset(x + (long)s * n, 0, sizeof(cplx) * n);
    }
    memcpy(r, b, sizeof(cplx) * n);
    double bb = norm2(b, n), rr = bb, alpha_prev = 1.0, beta_prev = 0.0;
    int k = 0;
    while (k < maxiter) {
        int any = 0;
        for (int s = 0; s < nshift; s++) any |= active[s];
        if (!any) break;
        const cplx *p0 = p + (long)s0 * n;
        apply_A(&op, p0, q);
        for (long i = 0; i < n; i++) q[i] += sigma[s0] * p0[i];
        double alpha = rr / creal(dot(p0, q, n));
        double zeta_new[nshift > 0 ? nshift : 1], alpha_s[nshift > 0 ? nshift : 1];
        for (int s = 0; s < nshift; s++) {
            double d = sigma[s] - sigma[s0];
            double den = alpha_prev * zeta_old[s] * (1.0 + alpha * d) +
                         alpha * beta_prev * (zeta_old[s] - zeta[s]);
            zeta_new[s] = zeta[s] * zeta_old[s] * alpha_prev / den;
            alpha_s[s] = alpha * zeta_new[s] / zeta[s];
        }
        for (int s = 0; s < nshift; s++)
            if (active[s]) {
                cplx *xs = x + (long)s * n, *ps = p + (long)s * n;
                for (long i = 0; i < n; i++) xs[i] += alpha_s[s] * ps[i];
            }
        for (long i = 0; i < n; i++) r[i] -= alpha * q[i];
        double rr_new = norm2(r, n);
        double beta = rr_new / rr;
        for (int s = 0; s < nshift; s++) {
            if (active[s]) {
                double ratio = zeta_new[s] / zeta[s];
                double beta_s = beta * ratio * ratio;
                cplx *ps = p + (long)s * n;
                for (long i = 0; i < n; i++) ps[i] = zeta_new[s] * r[i] + beta_s * ps[i];
            }
            zeta_old[s] = zeta[s];
            zeta[s] = zeta_new[s];
        }
        rr = rr_new;
        alpha_prev = alpha;
        beta_prev = beta;
        k++;
        for (int s = 0; s < nshift; s++)
            if (active[s] && fabs(zeta[s]) * sqrt(rr) <= tol[s] * sqrt(bb)) active[s] = 0;
    }
    stats[0] = k;
    int ok = 1;
    for (int s = 0; s < nshift; s++) {
        cplx *xs = x + (long)s * n;
        apply_A(&op, xs, q);
        for (long i = 0; i < n; i++) q[i] = b[i] - q[i] - sigma[s] * xs[i];
        stats[1 + s] = sqrt(norm2(q, n) / bb);
        if (stats[1 + s] > tol[s]) ok = 0;
    }
    free(r); free(q); free(p); free(op.tmp); free(zeta); free(zeta_old); free(active);
    return ok ? 0 : 1;
}

/* ------------------------------------------------------------------ learned preconditioner */

/*
 * Gauge-covariant parallel-transport network (not in the paper; its definition):
 *   layer l maps C_in -> C_out complex channels on the full lattice,
 *     psi'_{c'}(x) = sum_tap sum_c w[tap][c'][c] (T_tap psi_c)(x),
 *   taps: 0 = identity; 1 + 2mu + s = one hop, 9 + 2mu + s = three hops, s = 0 forward,
 *   s = 1 backward, with the transports of the Dslash stencil:
 *     T_{1+2mu}   psi(x) = X_mu(x) psi(x+mu)          T_{2+2mu}  psi(x) = X_mu(x-mu)^+ psi(x-mu)
 *     T_{9+2mu}   psi(x) = W_mu(x) psi(x+3mu)         T_{10+2mu} psi(x) = W_mu(x-3mu)^+ psi(x-3mu)
 *   each multiplied by eta_mu(x) and the hop's time boundary sign (unless `phased`),
 *   so that D = sum_mu (T_{1+2mu} - T_{2+2mu} + T_{9+2mu} - T_{10+2mu}).
 * Fields are [channel][V][3] complex in canonical order; weights of a layer are
 * [17][C_out][C_in] complex.  The adjoint of T_{forward} is T_{backward} of the same
 * direction and length.
 */
#define NTAP 17

static void transport(const lattice *L, const cplx *fat, const cplx *lng, int phased, int tap,
                      const cplx *in_full, const int x[4], cplx out[3])
{
    if (tap == 0) {
        const cplx *v = in_full + eo_index(L, x) * 3;
        for (int i = 0; i < 3; i++) out[i] = v[i];
        return;
    }
    int k = tap - 1, three = k >= 8;
    k &= 7;
    int mu = k >> 1, back = k & 1, len = three ? 3 : 1;
    const cplx *links = three ? lng : fat;
    int y[4];
    double bc = hop(L, x, mu, back ? -len : len, y);
    const cplx *v = in_full + eo_index(L, y) * 3;
    if (back) matvec_dag(link_at(L, links, mu, y), v, out);
    else matvec(link_at(L, links, mu, x), v, out);
    double s = phased ? 1.0 : eta(mu, x) * bc;
    for (int i = 0; i < 3; i++) out[i] *= s;
}

static int adjoint_tap(int tap)
{
    if (tap == 0) return 0;
    return ((tap - 1) ^ 1) + 1;
}

/* one layer: out[C_out][V][3] = sum_tap sum_c w[tap][c'][c] T_tap in[c] */
void ho_net_layer(const int dims[4], const double *fat, const double *lng, int phased, int cin,
                  int cout, const double *w, const double *in, double *out)
{
    lattice L = make_lattice(dims);
    const cplx *W = (const cplx *)w, *src = (const cplx *)in;
    cplx *dst = (cplx *)out;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < L.V; i++) {
        int x[4];
        coords_of(&L, i, x);
        cplx acc[cout > 0 ? cout : 1][3];
        memset(acc, 0, sizeof acc);
        for (int tap = 0; tap < NTAP; tap++)
            for (int c = 0; c < cin; c++) {
                cplx t[3];
                transport(&L, (const cplx *)fat, (const cplx *)lng, phased, tap,
                          src + (long)c * L.V * 3, x, t);
                for (int co = 0; co < cout; co++) {
                    cplx wt = W[((long)tap * cout + co) * cin + c];
                    for (int j = 0; j < 3; j++) acc[co][j] += wt * t[j];
                }
            }
        for (int co = 0; co < cout; co++)
            for (int j = 0; j < 3; j++) dst[((long)co * L.V + i) * 3 + j] = acc[co][j];
    }
}

/*
 * Backward of one layer for a real loss, with complex gradients g = dL/dRe + i dL/dIm:
 *   grad_in[c](x)      = sum_tap sum_c' conj(w[tap][c'][c]) (T_tap^+ g_out[c'])(x)
 *   grad_w[tap][c'][c] = sum_x sum_colour conj((T_tap in[c])(x)) g_out[c'](x)
 * grad_in may be NULL.
 */
void ho_net_layer_backward(const int dims[4], const double *fat, const double *lng, int phased,
                           int cin, int cout, const double *w, const double *in,
                           const double *gout, double *gin, double *gw)
{
    lattice L = make_lattice(dims);
    const cplx *W = (const cplx *)w, *src = (const cplx *)in, *g = (const cplx *)gout;
    cplx *GW = (cplx *)gw;
    for (int tap = 0; tap < NTAP; tap++)
        for (int co = 0; co < cout; co++)
            for (int c = 0; c < cin; c++) {
                double re = 0, im = 0;
#pragma omp parallel for reduction(+ : re, im) schedule(static)
                for (long i = 0; i < L.V; i++) {
                    int x[4];
                    cplx t[3];
                    coords_of(&L, i, x);
                    transport(&L, (const cplx *)fat, (const cplx *)lng, phased, tap,
                              src + (long)c * L.V * 3, x, t);
                    const cplx *gv = g + ((long)co * L.V + i) * 3;
                    cplx sacc = conj(t[0]) * gv[0] + conj(t[1]) * gv[1] + conj(t[2]) * gv[2];
                    re += creal(sacc);
                    im += cimag(sacc);
                }
                GW[((long)tap * cout + co) * cin + c] = re + I * im;
            }
    if (!gin) return;
    cplx *GI = (cplx *)gin;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < L.V; i++) {
        int x[4];
        coords_of(&L, i, x);
        for (int c = 0; c < cin; c++) {
            cplx acc[3] = {0, 0, 0};
            for (int tap = 0; tap < NTAP; tap++)
                for (int co = 0; co < cout; co++) {
                    cplx t[3];
                    transport(&L, (const cplx *)fat, (const cplx *)lng, phased, adjoint_tap(tap),
                              g + (long)co * L.V * 3, x, t);
                    cplx wc = conj(W[((long)tap * cout + co) * cin + c]);
                    for (int j = 0; j < 3; j++) acc[j] += wc * t[j];
                }
            for (int j = 0; j < 3; j++) GI[((long)c * L.V + i) * 3 + j] = acc[j];
        }
    }
}

/*
 * Whole network K(b): b on even sites (odd sites zero) -> layers -> restricted to even
 * sites.  chans[0..nlayer] are the channel counts (chans[0] = chans[nlayer] = 1);
 * weights are the layers' [17][C_out][C_in] blocks concatenated.
 */
static long layer_weights(const int *chans, int l) { return (long)NTAP * chans[l + 1] * chans[l]; }

void ho_net_apply(const int dims[4], const double *fat, const double *lng, int phased,
                  int nlayer, const int *chans, const double *w, const double *b_even,
                  double *z_even)
{
    lattice L = make_lattice(dims);
    int cmax = 1;
    for (int l = 0; l <= nlayer; l++) if (chans[l] > cmax) cmax = chans[l];
    cplx *a = calloc((size_t)cmax * L.V * 3, sizeof(cplx));
    cplx *bnext = calloc((size_t)cmax * L.V * 3, sizeof(cplx));
    memcpy(a, b_even, sizeof(cplx) * L.Vh * 3);
    const cplx *wl = (const cplx *)w;
    for (int l = 0; l < nlayer; l++) {
        ho_net_layer(dims, fat, lng, phased, chans[l], chans[l + 1], (const double *)wl,
                     (const double *)a, (double *)bnext);
        wl += layer_weights(chans, l);
        cplx *t = a; a = bnext; bnext = t;
    }
    memcpy(z_even, a, sizeof(cplx) * L.Vh * 3);
    free(a); free(bnext);
}

/*
 * Loss and gradient for one (b, x) pair: L = |K(b) - x|^2 / |x|^2 (even sites),
 * grad (complex convention) for every weight, written to gw (same layout as w).
 */
double ho_net_loss_grad(const int dims[4], const double *fat, const double *lng, int phased,
                        int nlayer, const int *chans, const double *w, const double *b_even,
                        const double *x_even, double *gw)
{
    lattice L = make_lattice(dims);
    long fs = L.V * 3;
    cplx **act = malloc(sizeof(cplx *) * (nlayer + 1));
    for (int l = 0; l <= nlayer; l++) act[l] = calloc((size_t)chans[l] * fs, sizeof(cplx));
    memcpy(act[0], b_even, sizeof(cplx) * L.Vh * 3);
    const cplx *wl = (const cplx *)w;
    for (int l = 0; l < nlayer; l++) {
        ho_net_layer(dims, fat, lng, phased, chans[l], chans[l + 1], (const double *)wl,
                     (const double *)act[l], (double *)act[l + 1]);
        wl += layer_weights(chans, l);
    }
    const cplx *xe = (const cplx *)x_even;
    double xx = 0, loss = 0;
    cplx *g = calloc((size_t)fs, sizeof(cplx));
    for (long i = 0; i < L.Vh * 3; i++) {
        cplx d = act[nlayer][i] - xe[i];
        loss += creal(conj(d) * d);
        xx += creal(conj(xe[i]) * xe[i]);
    }
    for (long i = 0; i < L.Vh * 3; i++) g[i] = 2.0 * (act[nlayer][i] - xe[i]) / xx;
    long off = 0;
    for (int l = 0; l < nlayer; l++) off += layer_weights(chans, l);
    for (int l = nlayer - 1; l >= 0; l--) {
        off -= layer_weights(chans, l);
        cplx *gin = l > 0 ? calloc((size_t)chans[l] * fs, sizeof(cplx)) : NULL;
        ho_net_layer_backward(dims, fat, lng, phased, chans[l], chans[l + 1],
                              (const double *)((const cplx *)w + off), (const double *)act[l],
                              (const double *)g, (double *)gin, (double *)((cplx *)gw + off));
        free(g);
        g = gin;
    }
    for (int l = 0; l <= nlayer; l++) free(act[l]);
    free(act);
    return loss / xx;
}

/* ------------------------------------------------------------------ flexible CG */

/*
 * Flexible (inexact-preconditioner) CG with the Polak-Ribiere beta, <a, b> = sum conj(a) b:
 *   r = b - A x; z = K r; p = z
 *   repeat: alpha = conj(<r, z>) / <p, A p>;  x += alpha p;  r_new = r - alpha A p
 *           z_new = K r_new;  beta = <r_new - r, z_new> / <r, z>;  p = z_new + beta p
 * until |r| <= tol |b|.  K is the network above (nlayer > 0) or the identity (nlayer = 0).
 * alpha minimises the A-norm of the error along p: alpha = <p, r> / <p, A p>, and
 * <p, r> = <z, r> = conj(<r, z>) because r is orthogonal to the previous direction; beta
 * makes the new direction A-orthogonal to p.  For a Hermitian K, <r, z> is real.
 * stats: [iterations, iterated |r|/|b|, recomputed |b - A x|/|b|].
 */
int ho_fcg(const int dims[4], const double *fat, const double *lng, int phased, double m,
           int nlayer, const int *chans, const double *w, const double *bv, double *xv,
           double tol, int maxiter, double stats[3])
{
    normal_op op = {make_lattice(dims), (const cplx *)fat, (const cplx *)lng, phased, m, NULL};
    long n = op.L.Vh * 3;
    const cplx *b = (const cplx *)bv;
    cplx *x = (cplx *)xv;
    cplx *r = malloc(sizeof(cplx) * n), *rn = malloc(sizeof(cplx) * n), *z = malloc(sizeof(cplx) * n);
    cplx *p = malloc(sizeof(cplx) * n), *Ap = malloc(sizeof(cplx) * n), *dr = malloc(sizeof(cplx) * n);
    op.tmp = malloc(sizeof(cplx) * n);
#define APPLY_K(src, dst) \
    do { \
        if (nlayer > 0) ho_net_apply(dims, fat, lng, phased, nlayer, chans, w, (const double *)(src), (double *)(dst)); \
        else memcpy((dst), (src), sizeof(cplx) * n); \
    } while (0)
    apply_A(&op, x, Ap);
    for (long i = 0; i < n; i++) r[i] = b[i] - Ap[i];
    APPLY_K(r, z);
    memcpy(p, z, sizeof(cplx) * n);
    double bb = norm2(b, n), rr = norm2(r, n);
    cplx rz = dot(r, z, n);
    int k = 0;
    while (k < maxiter && rr > tol * tol * bb) {
        apply_A(&op, p, Ap);
        cplx alpha = conj(rz) / creal(dot(p, Ap, n));
        for (long i = 0; i < n; i++) {
            x[i] += alpha * p[i];
            rn[i] = r[i] - alpha * Ap[i];
            dr[i] = rn[i] - r[i];
        }
        APPLY_K(rn, z);
        cplx beta = dot(dr, z, n) / rz;
        for (long i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
        memcpy(r, rn, sizeof(cplx) * n);
        rr = norm2(r, n);
        rz = dot(r, z, n);
        k++;
    }
#undef APPLY_K
    apply_A(&op, x, Ap);
    for (long i = 0; i < n; i++) r[i] = b[i] - Ap[i];
    stats[0] = k;
    stats[1] = sqrt(rr / bb);
    stats[2] = sqrt(norm2(r, n) / bb);
    free(r); free(rn); free(z); free(p); free(Ap); free(dr); free(op.tmp);
    return stats[2] <= tol ? 0 : 1;
}

/* dense preconditioner variant for the K = A^{-1} check: z = Kd r with Kd a dense
 * [3Vh][3Vh] complex matrix (row-major) */
int ho_fcg_dense(const int dims[4], const double *fat, const double *lng, int phased, double m,
                 const double *Kd, const double *bv, double *xv, double tol, int maxiter,
                 double stats[3])
{
    normal_op op = {make_lattice(dims), (const cplx *)fat, (const cplx *)lng, phased, m, NULL};
    long n = op.L.Vh * 3;
    const cplx *b = (const cplx *)bv, *K = (const cplx *)Kd;
    cplx *x = (cplx *)xv;
    cplx *r = malloc(sizeof(cplx) * n), *rn = malloc(sizeof(cplx) * n), *z = malloc(sizeof(cplx) * n);
    cplx *p = malloc(sizeof(cplx) * n), *Ap = malloc(sizeof(cplx) * n), *dr = malloc(sizeof(cplx) * n);
    op.tmp = malloc(sizeof(cplx) * n);
#define APPLY_KD(src, dst) \
    do { \
        for (long i_ = 0; i_ < n; i_++) { \
            cplx a_ = 0; \
            for (long j_ = 0; j_ < n; j_++) a_ += K[i_ * n + j_] * (src)[j_]; \
            (dst)[i_] = a_; \
        } \
    } while (0)
    apply_A(&op, x, Ap);
    for (long i = 0; i < n; i++) r[i] = b[i] - Ap[i];
    APPLY_KD(r, z);
    memcpy(p, z, sizeof(cplx) * n);
    double bb = norm2(b, n), rr = norm2(r, n);
    cplx rz = dot(r, z, n);
    int k = 0;
    while (k < maxiter && rr > tol * tol * bb) {
        apply_A(&op, p, Ap);
        cplx alpha = conj(rz) / creal(dot(p, Ap, n));
        for (long i = 0; i < n; i++) {
            x[i] += alpha * p[i];
            rn[i] = r[i] - alpha * Ap[i];
            dr[i] = rn[i] - r[i];
        }
        APPLY_KD(rn, z);
        cplx beta = dot(dr, z, n) / rz;
        for (long i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
        memcpy(r, rn, sizeof(cplx) * n);
        rr = norm2(r, n);
        rz = dot(r, z, n);
        k++;
    }
#undef APPLY_KD
    apply_A(&op, x, Ap);
    for (long i = 0; i < n; i++) r[i] = b[i] - Ap[i];
    stats[0] = k;
    stats[1] = sqrt(rr / bb);
    stats[2] = sqrt(norm2(r, n) / bb);
    free(r); free(rn); free(z); free(p); free(Ap); free(dr); free(op.tmp);
    return stats[2] <= tol ? 0 : 1;
}
