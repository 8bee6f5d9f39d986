/*
 * FP64 CPU oracle for the registration operator of the paper
 * "Parallel Prefix Algorithms for the Registration of Arbitrarily Long
 * Electron Micrograph Series" (arXiv 1712.02533).
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, double precision, written from the
 * paper's definitions; it shares no code with the CUDA path.  Only the tests,
 * the package's smoke check and the benchmark's CPU-baseline leg may call it.
 *
 * Conventions (readings of the paper where it is silent or ambiguous):
 *  - Level l is the vertex grid of (2^l+1)^2 nodes on Omega = [0,1]^2 (Section
 *    "Multilevel" picks the grid with a node on both borders); node (r, c) sits at
 *    x = (c h, r h), h = 2^-l; arrays are row-major, index r*n + c.
 *  - A deformation is stored as its displacement u = phi - id in Omega units,
 *    two planes: u[0..n^2) is the x_0 (column) part, u[n^2..2n^2) the x_1 (row)
 *    part.  phi maps reference coordinates into the template (f_1 o phi_01 = f_0,
 *    Section "Problem statement", the rectangle example with G = (0.25, 0)).
 *  - Sampling outside Omega clamps the coordinate to Omega; the derivative in a
 *    clamped coordinate is zero.  Inside, the bilinear cell is the one with
 *    index floor(p), capped at n-2 (the right/top cell on a node line).
 *
 * Parity status: every function here is pinned by tests/test_oracle_*.py
 * against closed forms, quadrature, finite differences, invariants or brute
 * force, except the Armijo decision sequence on real data, for which the paper
 * prints no worked numbers (parity unpinned for that sequence; the
 * surrounding functions are pinned).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

static double *dalloc(size_t n) { return (double *)calloc(n, sizeof(double)); }

/* Optional trace of every Armijo trial of orc_solve_level (for comparing
 * decision sequences in tests): records of 6 doubles
 * {n, iteration, tau, E(u + tau d) - E(u), sigma tau g^T d, accepted}.
 * One trace per host thread, so that operators solved on several threads at
 * once each record their own. */
static _Thread_local double *g_trace = NULL;
static _Thread_local long g_trace_cap = 0, g_trace_len = 0;

void orc_set_trace(double *buf, long cap)
{
    g_trace = buf;
    g_trace_cap = cap;
    g_trace_len = 0;
}

long orc_trace_len(void) { return g_trace_len; }

static void trace(int n, int it, double tau, double dE, double rhs, int acc)
{
    if (!g_trace || g_trace_len >= g_trace_cap) return;
    double *r = g_trace + 6 * g_trace_len++;
    r[0] = n;
    r[1] = it;
    r[2] = tau;
    r[3] = dE;
    r[4] = rhs;
    r[5] = acc;
}

/* ------------------------------------------------------------------------- */
/* Grids, embedding, restriction and prolongation (Section "Multilevel")     */
/* ------------------------------------------------------------------------- */

/* A 2^L x 2^L frame becomes the (2^L+1)^2 vertex grid of level L; the extra
 * last row and column repeat the frame's last row and column. */
void orc_embed(const float *frame, int side, double *out)
{
    int n = side + 1;
    for (int r = 0; r < n; r++) {
        int rr = r < side ? r : side - 1;
        for (int c = 0; c < n; c++) {
            int cc = c < side ? c : side - 1;
            out[r * n + c] = (double)frame[rr * side + cc];
        }
    }
}

static int mirror(int i, int n)
{
    if (i < 0) return -i;
    if (i > n - 1) return 2 * (n - 1) - i;
    return i;
}

/* Restriction with the 1/16 [1 2 1; 2 4 2; 1 2 1] stencil (Section
 * "Multilevel"): coarse node (I, J) is the stencil average around fine node
 * (2I, 2J); fine indices past the boundary are mirrored. */
void orc_restrict(const double *fine, int nf, double *coarse)
{
    int nc = (nf + 1) / 2;
    static const double w[3] = {0.25, 0.5, 0.25};
    for (int I = 0; I < nc; I++)
        for (int J = 0; J < nc; J++) {
            double s = 0.0;
            for (int a = -1; a <= 1; a++)
                for (int b = -1; b <= 1; b++) {
                    int r = mirror(2 * I + a, nf), c = mirror(2 * J + b, nf);
                    s += w[a + 1] * w[b + 1] * fine[r * nf + c];
                }
            coarse[I * nc + J] = s;
        }
}

/* Prolongation I_l^{2l} (Section "Multilevel"): coarse nodes are copied, new
 * nodes get the bilinear interpolation of their coarse neighbours (2 on an
 * edge midpoint, 4 at a cell centre). */
void orc_prolong(const double *coarse, int nc, double *fine)
{
    int nf = 2 * nc - 1;
    for (int r = 0; r < nf; r++)
        for (int c = 0; c < nf; c++) {
            int I = r / 2, J = c / 2;
            double v;
            if (r % 2 == 0 && c % 2 == 0)
                v = coarse[I * nc + J];
            else if (r % 2 == 0)
                v = 0.5 * (coarse[I * nc + J] + coarse[I * nc + J + 1]);
            else if (c % 2 == 0)
                v = 0.5 * (coarse[I * nc + J] + coarse[(I + 1) * nc + J]);
            else
                v = 0.25 * (coarse[I * nc + J] + coarse[I * nc + J + 1] +
                            coarse[(I + 1) * nc + J] + coarse[(I + 1) * nc + J + 1]);
            fine[r * nf + c] = v;
        }
}

/* ------------------------------------------------------------------------- */
/* FE operators (Section "Spatial discretization")                           */
/* ------------------------------------------------------------------------- */

/* 1D piecewise-linear mass matrix entry  int psi_i psi_j  on a uniform grid. */
static double m1(int i, int j, int n, double h)
{
    if (i == j) return (i == 0 || i == n - 1) ? h / 3.0 : 2.0 * h / 3.0;
    if (i - j == 1 || j - i == 1) return h / 6.0;
    return 0.0;
}

/* 1D stiffness entry  int psi_i' psi_j'. */
static double k1(int i, int j, int n, double h)
{
    if (i == j) return (i == 0 || i == n - 1) ? 1.0 / h : 2.0 / h;
    if (i - j == 1 || j - i == 1) return -1.0 / h;
    return 0.0;
}

/* out = (A_row (x) A_col) v for tensor-product bilinear basis functions
 * phi_(r,c)(x) = psi_c(x_0) psi_r(x_1): entry ((r,c),(a,b)) = A_row[r][a] A_col[c][b]. */
static void kron_apply(double (*arow)(int, int, int, double), double (*acol)(int, int, int, double),
                       const double *v, int n, double *out)
{
    double h = 1.0 / (n - 1);
    double *tmp = dalloc((size_t)n * n);
    /* along columns (x_0): tmp[r][c] = sum_b acol(c, b) v[r][b] */
    for (int r = 0; r < n; r++)
        for (int c = 0; c < n; c++) {
            double s = 0.0;
            for (int b = c - 1; b <= c + 1; b++)
                if (b >= 0 && b < n) s += acol(c, b, n, h) * v[r * n + b];
            tmp[r * n + c] = s;
        }
    /* along rows (x_1) */
    for (int r = 0; r < n; r++)
        for (int c = 0; c < n; c++) {
            double s = 0.0;
            for (int a = r - 1; a <= r + 1; a++)
                if (a >= 0 && a < n) s += arow(r, a, n, h) * tmp[a * n + c];
            out[r * n + c] = s;
        }
    free(tmp);
}

/* Mass matrix M_ij = int phi_i phi_j = M1 (x) M1. */
void orc_mass_apply(const double *v, int n, double *out) { kron_apply(m1, m1, v, n, out); }

/* Stiffness K_ij = int grad phi_i . grad phi_j = K1 (x) M1 + M1 (x) K1; it
 * discretises the Dirichlet energy int |D v|^2 = v^T K v. */
void orc_stiff_apply(const double *v, int n, double *out)
{
    double *a = dalloc((size_t)n * n);
    kron_apply(k1, m1, v, n, out); /* d/dx_1 part: K1 along rows */
    kron_apply(m1, k1, v, n, a);   /* d/dx_0 part: K1 along columns */
    for (int i = 0; i < n * n; i++) out[i] += a[i];
    free(a);
}

/* Lumped weights w = M 1 (so that the mean is w^T F). */
void orc_lumped(int n, double *w)
{
    double *one = dalloc((size_t)n * n);
    for (int i = 0; i < n * n; i++) one[i] = 1.0;
    orc_mass_apply(one, n, w);
    free(one);
}

static double dot(const double *a, const double *b, size_t n)
{
    double s = 0.0;
    for (size_t i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

/* ------------------------------------------------------------------------- */
/* Warping (T o phi sampled at the nodes)                                    */
/* ------------------------------------------------------------------------- */

/* Bilinear interpolant of nodal values T at the point (x0, x1) in Omega
 * units, clamped to Omega; d0/d1 (nullable) get its partial derivatives in
 * Omega units, zero in a clamped coordinate. */
double orc_interp(const double *T, int n, double x0, double x1, double *d0, double *d1)
{
    double h = 1.0 / (n - 1);
    int cl0 = 0, cl1 = 0;
    if (x0 < 0.0) { x0 = 0.0; cl0 = 1; }
    if (x0 > 1.0) { x0 = 1.0; cl0 = 1; }
    if (x1 < 0.0) { x1 = 0.0; cl1 = 1; }
    if (x1 > 1.0) { x1 = 1.0; cl1 = 1; }
    double p0 = x0 * (n - 1), p1 = x1 * (n - 1);
    int j0 = (int)floor(p0), j1 = (int)floor(p1);
    if (j0 > n - 2) j0 = n - 2;
    if (j1 > n - 2) j1 = n - 2;
    if (j0 < 0) j0 = 0;
    if (j1 < 0) j1 = 0;
    double f0 = p0 - j0, f1 = p1 - j1;
    double t00 = T[j1 * n + j0], t01 = T[j1 * n + j0 + 1];
    double t10 = T[(j1 + 1) * n + j0], t11 = T[(j1 + 1) * n + j0 + 1];
    double v = (1 - f1) * ((1 - f0) * t00 + f0 * t01) + f1 * ((1 - f0) * t10 + f0 * t11);
    if (d0) *d0 = cl0 ? 0.0 : ((1 - f1) * (t01 - t00) + f1 * (t11 - t10)) / h;
    if (d1) *d1 = cl1 ? 0.0 : ((1 - f0) * (t10 - t00) + f0 * (t11 - t01)) / h;
    return v;
}

/* That_i = T(x_i + u_i): nodal interpolation of the deformed template. */
void orc_warp(const double *T, int n, const double *u, double *That, double *dT)
{
    double h = 1.0 / (n - 1);
    size_t N = (size_t)n * n;
    for (int r = 0; r < n; r++)
        for (int c = 0; c < n; c++) {
            size_t i = (size_t)r * n + c;
            double d0, d1;
            That[i] = orc_interp(T, n, c * h + u[i], r * h + u[N + i], &d0, &d1);
            if (dT) {
                dT[i] = d0;
                dT[N + i] = d1;
            }
        }
}

/* ------------------------------------------------------------------------- */
/* Energy and gradient (Section "Image registration for electron microscopy",*/
/* the NCC and energy definitions, discretised as in "Spatial discretization")*/
/* ------------------------------------------------------------------------- */

/* E[phi] = -NCC[R, T o phi] + lambda/2 int |D(phi(x) - x)|^2.
 * Mean f_bar = w^T F, sigma_f^2 = (F - f_bar)^T M (F - f_bar),
 * NCC = (R - R_bar)^T M (That - T_bar) / (sigma_R sigma_T).
 * parts (nullable, 6): NCC, regulariser, R_bar, sigma_R, T_bar, sigma_T. */
double orc_energy(const double *R, const double *T, int n, const double *u, double lambda,
                  double *parts)
{
    size_t N = (size_t)n * n;
    double *w = dalloc(N), *Th = dalloc(N), *Rc = dalloc(N), *Tc = dalloc(N), *Mv = dalloc(N);
    orc_lumped(n, w);
    orc_warp(T, n, u, Th, NULL);
    double Rbar = dot(w, R, N), Tbar = dot(w, Th, N);
    for (size_t i = 0; i < N; i++) {
        Rc[i] = R[i] - Rbar;
        Tc[i] = Th[i] - Tbar;
    }
    orc_mass_apply(Rc, n, Mv);
    double sR = sqrt(dot(Rc, Mv, N));
    double cross = dot(Mv, Tc, N);
    orc_mass_apply(Tc, n, Mv);
    double sT = sqrt(dot(Tc, Mv, N));
    double ncc = cross / (sR * sT);
    double reg = 0.0;
    for (int ch = 0; ch < 2; ch++) {
        orc_stiff_apply(u + ch * N, n, Mv);
        reg += dot(u + ch * N, Mv, N);
    }
    reg *= 0.5 * lambda;
    if (parts) {
        parts[0] = ncc;
        parts[1] = reg;
        parts[2] = Rbar;
        parts[3] = sR;
        parts[4] = Tbar;
        parts[5] = sT;
    }
    free(w);
    free(Th);
    free(Rc);
    free(Tc);
    free(Mv);
    return -ncc + reg;
}

/* g = dE/du (Euclidean gradient of the discrete energy, Omega units):
 *   dNCC/dThat = M Rc/(sigma_R sigma_T) - NCC * M Tc / sigma_T^2,
 *   g_{i,c} = -(dNCC/dThat)_i  d_c T(x_i + u_i) + lambda (K u_c)_i.
 * This is the first variation E' of the gradient-flow equation (Section
 * "Gradient flow"), exact for the discrete E away from cell lines. */
void orc_gradient(const double *R, const double *T, int n, const double *u, double lambda,
                  double *g)
{
    size_t N = (size_t)n * n;
    double *w = dalloc(N), *Th = dalloc(N), *dT = dalloc(2 * N), *Rc = dalloc(N), *Tc = dalloc(N);
    double *MRc = dalloc(N), *MTc = dalloc(N), *Ku = dalloc(N);
    orc_lumped(n, w);
    orc_warp(T, n, u, Th, dT);
    double Rbar = dot(w, R, N), Tbar = dot(w, Th, N);
    for (size_t i = 0; i < N; i++) {
        Rc[i] = R[i] - Rbar;
        Tc[i] = Th[i] - Tbar;
    }
    orc_mass_apply(Rc, n, MRc);
    orc_mass_apply(Tc, n, MTc);
    double sR = sqrt(dot(Rc, MRc, N)), sT = sqrt(dot(Tc, MTc, N));
    double ncc = dot(MRc, Tc, N) / (sR * sT);
    for (int ch = 0; ch < 2; ch++) {
        orc_stiff_apply(u + ch * N, n, Ku);
        for (size_t i = 0; i < N; i++) {
            double dncc = MRc[i] / (sR * sT) - ncc * MTc[i] / (sT * sT);
            g[ch * N + i] = -dncc * dT[ch * N + i] + lambda * Ku[i];
        }
    }
    free(w);
    free(Th);
    free(dT);
    free(Rc);
    free(Tc);
    free(MRc);
    free(MTc);
    free(Ku);
}

/* ------------------------------------------------------------------------- */
/* Gradient flow with the Armijo rule with widening (Section "Gradient flow")*/
/* ------------------------------------------------------------------------- */

/* ------------------------------------------------------------------------- */
/* H1-type smoother (Section "Gradient flow": A^{-1} smooths the first        */
/* variation in the non-rigid registration)                                   */
/* ------------------------------------------------------------------------- */

/* 1D H1 Gram matrix M_s = M1 + (s^2/2) K1 with s = smooth * h (the smoother's
 * width in grid spacings of the level): int psi_i psi_j + s^2/2 int psi_i' psi_j'. */
static _Thread_local double m1s_smooth;
static double m1s(int i, int j, int n, double h)
{
    double s = m1s_smooth * h;
    return m1(i, j, n, h) + 0.5 * s * s * k1(i, j, n, h);
}

/* out = (M_s (x) M_s) v: the tensor-product H1 Gram matrix applied to one
 * plane of nodal values. */
void orc_smooth_matvec(int n, double smooth, const double *v, double *out)
{
    m1s_smooth = smooth;
    kron_apply(m1s, m1s, v, n, out);
}

/* Solve the tridiagonal 1D system M_s x = b along one line (stride st): the
 * plain Thomas elimination. */
static void smooth_line(int n, double h, double smooth, const double *b, double *x, size_t st)
{
    double s = smooth * h, c = 0.5 * s * s;
    double *cp = dalloc((size_t)n), *dp = dalloc((size_t)n);
    for (int i = 0; i < n; i++) {
        double diag = m1(i, i, n, h) + c * k1(i, i, n, h);
        double lo = i > 0 ? m1(i, i - 1, n, h) + c * k1(i, i - 1, n, h) : 0.0;
        double up = i < n - 1 ? m1(i, i + 1, n, h) + c * k1(i, i + 1, n, h) : 0.0;
        double den = diag - (i > 0 ? lo * cp[i - 1] : 0.0);
        cp[i] = up / den;
        dp[i] = (b[(size_t)i * st] - (i > 0 ? lo * dp[i - 1] : 0.0)) / den;
    }
    x[(size_t)(n - 1) * st] = dp[n - 1];
    for (int i = n - 2; i >= 0; i--) x[(size_t)i * st] = dp[i] - cp[i] * x[(size_t)(i + 1) * st];
    free(cp);
    free(dp);
}

/* d = -(M_s (x) M_s)^{-1} g for both planes of g: since the matrix is a
 * Kronecker product, its inverse is M_s^{-1} (x) M_s^{-1}, i.e. one 1D solve
 * along every row, then one along every column. */
void orc_smooth_apply(int n, double smooth, const double *g, double *d)
{
    double h = 1.0 / (n - 1);
    size_t N = (size_t)n * n;
    double *t = dalloc(N);
    for (int ch = 0; ch < 2; ch++) {
        const double *gc = g + ch * N;
        double *dc = d + ch * N;
        for (int r = 0; r < n; r++) smooth_line(n, h, smooth, gc + (size_t)r * n, t + (size_t)r * n, 1);
        for (int c = 0; c < n; c++) smooth_line(n, h, smooth, t + c, dc + c, (size_t)n);
        for (size_t i = 0; i < N; i++) dc[i] = -dc[i];
    }
    free(t);
}

/* Forward Euler step phi^{k+1} = phi^k - tau A^{-1} E'[phi^k] with the
 * smoother A = diag(w) (lumped mass, an L2 gradient flow), i.e. direction
 * d = -g / w, or with p->smooth > 0 the tensor-product H1 Gram matrix
 * A = M_s (x) M_s (orc_smooth_apply).  Step size: start from the previous accepted tau (tau_init at the
 * start of the level); if the Armijo condition
 *     E(u + tau d) - E(u) <= sigma tau g^T d
 * holds, keep doubling while it still holds and 2 tau <= tau_max; otherwise
 * halve until it holds, giving up below tau_min.  Stop when the energy
 * decrease is below epsilon * max(1, |E|) or after iter_max iterations
 * (Algorithm "Multilevel gradient flow" stopping criteria). */
int orc_solve_level(const double *R, const double *T, int n, double *u, const orc_params *p,
                    orc_level_stats *st)
{
    size_t N = (size_t)n * n;
    double *w = dalloc(N), *g = dalloc(2 * N), *d = dalloc(2 * N), *ut = dalloc(2 * N);
    orc_lumped(n, w);
    int iters = 0, trials = 0, status = ORC_MAXITER;
    double E0 = orc_energy(R, T, n, u, p->lambda, NULL);
    double Estart = E0;
    double tau = p->tau_init;
    if (!isfinite(E0)) status = ORC_NONFINITE;
    for (int it = 0; status != ORC_NONFINITE && it < p->iter_max; it++) {
        orc_gradient(R, T, n, u, p->lambda, g);
        iters++;
        double slope = 0.0;
        if (p->smooth > 0.0) orc_smooth_apply(n, p->smooth, g, d);
        else
            for (size_t i = 0; i < 2 * N; i++) d[i] = -g[i] / w[i % N];
        for (size_t i = 0; i < 2 * N; i++) slope += g[i] * d[i];
        if (!(slope < 0.0)) {
            status = (slope == 0.0) ? ORC_ZERO_GRADIENT : ORC_NONFINITE;
            break;
        }
#define TRIAL(t_, E_)                                                   \
    do {                                                                \
        for (size_t i_ = 0; i_ < 2 * N; i_++) ut[i_] = u[i_] + (t_) * d[i_]; \
        (E_) = orc_energy(R, T, n, ut, p->lambda, NULL);                \
        trials++;                                                       \
    } while (0)
        double E1;
        int stalled = 0;
        TRIAL(tau, E1);
        int ok = E1 - E0 <= p->armijo_sigma * tau * slope;
        trace(n, it, tau, E1 - E0, p->armijo_sigma * tau * slope, ok);
        if (ok) {
            for (;;) {
                double t2 = 2.0 * tau, Et;
                if (t2 > p->tau_max) break;
                TRIAL(t2, Et);
                int ok2 = Et - E0 <= p->armijo_sigma * t2 * slope;
                trace(n, it, t2, Et - E0, p->armijo_sigma * t2 * slope, ok2);
                if (ok2) {
                    tau = t2;
                    E1 = Et;
                } else {
                    break;
                }
            }
        } else {
            for (;;) {
                tau = 0.5 * tau;
                if (tau < p->tau_min) {
                    stalled = 1;
                    break;
                }
                TRIAL(tau, E1);
                int ok3 = E1 - E0 <= p->armijo_sigma * tau * slope;
                trace(n, it, tau, E1 - E0, p->armijo_sigma * tau * slope, ok3);
                if (ok3) break;
            }
        }
#undef TRIAL
        if (stalled) {
            status = ORC_LS_STALLED;
            break;
        }
        for (size_t i = 0; i < 2 * N; i++) u[i] += tau * d[i];
        double dec = E0 - E1, scale = fabs(E0) > 1.0 ? fabs(E0) : 1.0;
        E0 = E1;
        if (dec < p->epsilon * scale) {
            status = ORC_CONVERGED;
            break;
        }
    }
    if (st) {
        st->iters = iters;
        st->trials = trials;
        st->status = status;
        st->E_start = Estart;
        st->E = E0;
        st->tau = tau;
    }
    free(w);
    free(g);
    free(d);
    free(ut);
    return status;
}

/* ------------------------------------------------------------------------- */
/* Function A: multilevel gradient flow (Algorithm "Multilevel gradient flow")*/
/* ------------------------------------------------------------------------- */

/* R, T: nodal grids of level L (n = 2^L + 1).  u_init: level-L displacement
 * (Omega units) or NULL for the identity.  Coarse grids for R, T and the
 * initial displacement are produced by restriction down to m0 = L-n_levels+1;
 * the flow is solved from m0 up to L, prolongating between levels.
 * u_out: level-L result.  st: n_levels entries, coarsest first. */
int orc_register(const double *R, const double *T, int L, const double *u_init,
                 const orc_params *p, double *u_out, orc_level_stats *st)
{
    int nl = p->n_levels;
    if (nl < 1 || nl > L + 1) return -1;
    int m0 = L - nl + 1;
    double *Rl[32], *Tl[32], *ul[32];
    int nn[32];
    for (int l = m0; l <= L; l++) {
        nn[l] = (1 << l) + 1;
        size_t N = (size_t)nn[l] * nn[l];
        Rl[l] = dalloc(N);
        Tl[l] = dalloc(N);
        ul[l] = dalloc(2 * N);
    }
    size_t NL = (size_t)nn[L] * nn[L];
    memcpy(Rl[L], R, NL * sizeof(double));
    memcpy(Tl[L], T, NL * sizeof(double));
    if (u_init) memcpy(ul[L], u_init, 2 * NL * sizeof(double));
    for (int l = L - 1; l >= m0; l--) {
        orc_restrict(Rl[l + 1], nn[l + 1], Rl[l]);
        orc_restrict(Tl[l + 1], nn[l + 1], Tl[l]);
        if (u_init) {
            size_t Nf = (size_t)nn[l + 1] * nn[l + 1], Nc = (size_t)nn[l] * nn[l];
            orc_restrict(ul[l + 1], nn[l + 1], ul[l]);
            orc_restrict(ul[l + 1] + Nf, nn[l + 1], ul[l] + Nc);
        }
    }
    int worst = ORC_CONVERGED;
    for (int l = m0; l <= L; l++) {
        int s = orc_solve_level(Rl[l], Tl[l], nn[l], ul[l], p, st ? &st[l - m0] : NULL);
        if (s == ORC_NONFINITE) worst = ORC_NONFINITE;
        if (l < L) {
            size_t Nf = (size_t)nn[l + 1] * nn[l + 1], Nc = (size_t)nn[l] * nn[l];
            orc_prolong(ul[l], nn[l], ul[l + 1]);
            orc_prolong(ul[l] + Nc, nn[l], ul[l + 1] + Nf);
        } else if (worst != ORC_NONFINITE) {
            worst = s;
        }
    }
    memcpy(u_out, ul[L], 2 * NL * sizeof(double));
    for (int l = m0; l <= L; l++) {
        free(Rl[l]);
        free(Tl[l]);
        free(ul[l]);
    }
    return worst;
}

/* ------------------------------------------------------------------------- */
/* Composition and function B (Section "Registration for series of images")  */
/* ------------------------------------------------------------------------- */

/* phi_ik = phi_jk o phi_ij (phi_ij applied first): in displacements
 * u_ik(x) = u_ij(x) + u_jk(x + u_ij(x)), u_jk read by bilinear interpolation
 * with the point clamped to Omega. */
void orc_compose(const double *u_ij, const double *u_jk, int n, double *out)
{
    double h = 1.0 / (n - 1);
    size_t N = (size_t)n * n;
    for (int r = 0; r < n; r++)
        for (int c = 0; c < n; c++) {
            size_t i = (size_t)r * n + c;
            double y0 = c * h + u_ij[i], y1 = r * h + u_ij[N + i];
            out[i] = u_ij[i] + orc_interp(u_jk, n, y0, y1, NULL, NULL);
            out[N + i] = u_ij[N + i] + orc_interp(u_jk + N, n, y0, y1, NULL, NULL);
        }
}

/* A batch of independent operator applications.  Per op: R, T (level-L grids
 * of that op's series), L, and the initial guess: both left and right given
 * -> B = A(R, T, right o left); only left -> A(R, T, left); none -> A(R, T, I).
 * Independent ops run in parallel over host threads. */
void orc_apply_batch(int n_ops, const double *const *R, const double *const *T, const int32_t *L,
                     const double *const *left, const double *const *right, double *const *out,
                     const orc_params *p, int32_t *status, int32_t *iters, int32_t *trials,
                     double *energy)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int o = 0; o < n_ops; o++) {
        int n = (1 << L[o]) + 1;
        size_t N = (size_t)n * n;
        double *init = NULL;
        if (left[o] && right[o]) {
            init = dalloc(2 * N);
            orc_compose(left[o], right[o], n, init);
        } else if (left[o]) {
            init = dalloc(2 * N);
            memcpy(init, left[o], 2 * N * sizeof(double));
        }
        orc_level_stats st[32];
        int s = orc_register(R[o], T[o], L[o], init, p, out[o], st);
        int it = 0, tr = 0;
        for (int l = 0; l < p->n_levels; l++) {
            it += st[l].iters;
            tr += st[l].trials;
        }
        if (status) status[o] = s;
        if (iters) iters[o] = it;
        if (trials) trials[o] = tr;
        if (energy) energy[o] = st[p->n_levels - 1].E;
        free(init);
    }
}

/* ------------------------------------------------------------------------- */
/* Series averaging (Section "Introduction": the deformed frames              */
/* f_i o phi_{0,i} of an aligned series are averaged into one frame; Section   */
/* "Registration for series of images": the series averaging procedure)       */
/* ------------------------------------------------------------------------- */

/* avg = 1/m sum_k F_k o (id + u_k), nodal interpolation on the vertex grid of
 * n x n nodes: F_k are the m embedded frames (nodal values), u_k their
 * displacements in Omega units (two planes each; NULL = the identity). */
void orc_average(int m, const double *const *F, const double *const *u, int n, double *avg)
{
    double h = 1.0 / (n - 1);
    size_t N = (size_t)n * n;
    for (size_t i = 0; i < N; i++) avg[i] = 0.0;
    for (int k = 0; k < m; k++)
        for (int r = 0; r < n; r++)
            for (int c = 0; c < n; c++) {
                size_t i = (size_t)r * n + c;
                double x0 = c * h, x1 = r * h;
                if (u[k]) {
                    x0 += u[k][i];
                    x1 += u[k][N + i];
                }
                avg[i] += orc_interp(F[k], n, x0, x1, NULL, NULL);
            }
    for (size_t i = 0; i < N; i++) avg[i] /= m;
}

/* ------------------------------------------------------------------------- */
/* Rigid variant (Definition "Rigid transformation": phi(x) = R(alpha) x + t, */
/* rotation about the origin of Omega; Section "Gradient flow": the smoother  */
/* is applied only in the non-rigid registration; Algorithm "Multilevel       */
/* gradient flow": a rigid deformation is not restricted or prolongated)      */
/* ------------------------------------------------------------------------- */

/* Nodal displacement u(x) = R(alpha) x + t - x of theta = (alpha, t0, t1),
 * Omega units, two planes. */
void orc_rigid_field(const double *theta, int n, double *u)
{
    double h = 1.0 / (n - 1), ca = cos(theta[0]), sa = sin(theta[0]);
    size_t N = (size_t)n * n;
    for (int r = 0; r < n; r++)
        for (int c = 0; c < n; c++) {
            double x0 = c * h, x1 = r * h;
            u[(size_t)r * n + c] = ca * x0 - sa * x1 + theta[1] - x0;
            u[N + (size_t)r * n + c] = sa * x0 + ca * x1 + theta[2] - x1;
        }
}

double orc_rigid_energy(const double *R, const double *T, int n, const double *theta, double lambda)
{
    double *u = dalloc(2 * (size_t)n * n);
    orc_rigid_field(theta, n, u);
    double E = orc_energy(R, T, n, u, lambda, NULL);
    free(u);
    return E;
}

/* dE/dtheta_j = sum_i g_i . du_i/dtheta_j with g the nodal gradient of the
 * discrete energy (orc_gradient): du/dalpha = R'(alpha) x, du/dt_c = e_c. */
void orc_rigid_gradient(const double *R, const double *T, int n, const double *theta, double lambda, double *grad)
{
    size_t N = (size_t)n * n;
    double h = 1.0 / (n - 1), ca = cos(theta[0]), sa = sin(theta[0]);
    double *u = dalloc(2 * N), *g = dalloc(2 * N);
    orc_rigid_field(theta, n, u);
    orc_gradient(R, T, n, u, lambda, g);
    grad[0] = grad[1] = grad[2] = 0.0;
    for (int r = 0; r < n; r++)
        for (int c = 0; c < n; c++) {
            size_t i = (size_t)r * n + c;
            double x0 = c * h, x1 = r * h;
            grad[0] += g[i] * (-sa * x0 - ca * x1) + g[N + i] * (ca * x0 - sa * x1);
            grad[1] += g[i];
            grad[2] += g[N + i];
        }
    free(u);
    free(g);
}

/* Gradient descent on theta with the Armijo rule with widening of
 * orc_solve_level (direction d = -grad E, no smoother). */
int orc_rigid_solve_level(const double *R, const double *T, int n, double *theta, const orc_params *p,
                          orc_level_stats *st)
{
    int iters = 0, trials = 0, status = ORC_MAXITER;
    double E0 = orc_rigid_energy(R, T, n, theta, p->lambda), Estart = E0, tau = p->tau_init;
    if (!isfinite(E0)) status = ORC_NONFINITE;
    for (int it = 0; status != ORC_NONFINITE && it < p->iter_max; it++) {
        double g[3], d[3], th[3];
        orc_rigid_gradient(R, T, n, theta, p->lambda, g);
        iters++;
        double slope = 0.0;
        for (int j = 0; j < 3; j++) {
            d[j] = -g[j];
            slope += g[j] * d[j];
        }
        if (!(slope < 0.0)) {
            status = (slope == 0.0) ? ORC_ZERO_GRADIENT : ORC_NONFINITE;
            break;
        }
#define RTRIAL(t_, E_)                                                      \
    do {                                                                    \
        for (int j_ = 0; j_ < 3; j_++) th[j_] = theta[j_] + (t_) * d[j_];   \
        (E_) = orc_rigid_energy(R, T, n, th, p->lambda);                    \
        trials++;                                                           \
    } while (0)
        double E1;
        int stalled = 0;
        RTRIAL(tau, E1);
        int ok = E1 - E0 <= p->armijo_sigma * tau * slope;
        trace(n, it, tau, E1 - E0, p->armijo_sigma * tau * slope, ok);
        if (ok) {
            for (;;) {
                double t2 = 2.0 * tau, Et;
                if (t2 > p->tau_max) break;
                RTRIAL(t2, Et);
                int ok2 = Et - E0 <= p->armijo_sigma * t2 * slope;
                trace(n, it, t2, Et - E0, p->armijo_sigma * t2 * slope, ok2);
                if (!ok2) break;
                tau = t2;
                E1 = Et;
            }
        } else {
            for (;;) {
                tau = 0.5 * tau;
                if (tau < p->tau_min) {
                    stalled = 1;
                    break;
                }
                RTRIAL(tau, E1);
                int ok3 = E1 - E0 <= p->armijo_sigma * tau * slope;
                trace(n, it, tau, E1 - E0, p->armijo_sigma * tau * slope, ok3);
                if (ok3) break;
            }
        }
#undef RTRIAL
        if (stalled) {
            status = ORC_LS_STALLED;
            break;
        }
        for (int j = 0; j < 3; j++) theta[j] += tau * d[j];
        double dec = E0 - E1, scale = fabs(E0) > 1.0 ? fabs(E0) : 1.0;
        E0 = E1;
        if (dec < p->epsilon * scale) {
            status = ORC_CONVERGED;
            break;
        }
    }
    if (st) {
        st->iters = iters;
        st->trials = trials;
        st->status = status;
        st->E_start = Estart;
        st->E = E0;
        st->tau = tau;
    }
    return status;
}

/* Multilevel rigid registration: the images are restricted down to m0 as in
 * orc_register; the three parameters are carried from level to level as they
 * are (they do not depend on the grid). */
int orc_rigid_register(const double *R, const double *T, int L, const double *theta_init, const orc_params *p,
                       double *theta_out, orc_level_stats *st)
{
    int nl = p->n_levels;
    if (nl < 1 || nl > L + 1) return -1;
    int m0 = L - nl + 1;
    double *Rl[32], *Tl[32];
    int nn[32];
    for (int l = m0; l <= L; l++) {
        nn[l] = (1 << l) + 1;
        Rl[l] = dalloc((size_t)nn[l] * nn[l]);
        Tl[l] = dalloc((size_t)nn[l] * nn[l]);
    }
    memcpy(Rl[L], R, (size_t)nn[L] * nn[L] * sizeof(double));
    memcpy(Tl[L], T, (size_t)nn[L] * nn[L] * sizeof(double));
    for (int l = L - 1; l >= m0; l--) {
        orc_restrict(Rl[l + 1], nn[l + 1], Rl[l]);
        orc_restrict(Tl[l + 1], nn[l + 1], Tl[l]);
    }
    double th[3] = {0.0, 0.0, 0.0};
    if (theta_init) memcpy(th, theta_init, sizeof(th));
    int worst = ORC_CONVERGED;
    for (int l = m0; l <= L; l++) {
        int s = orc_rigid_solve_level(Rl[l], Tl[l], nn[l], th, p, st ? &st[l - m0] : NULL);
        if (s == ORC_NONFINITE) worst = ORC_NONFINITE;
        else if (l == L && worst != ORC_NONFINITE) worst = s;
    }
    memcpy(theta_out, th, sizeof(th));
    for (int l = m0; l <= L; l++) {
        free(Rl[l]);
        free(Tl[l]);
    }
    return worst;
}

/* phi_b o phi_a for rigid maps (phi_a applied first):
 * R(b0) (R(a0) x + ta) + tb = R(a0 + b0) x + R(b0) ta + tb. */
void orc_rigid_compose(const double *a, const double *b, double *out)
{
    double cb = cos(b[0]), sb = sin(b[0]);
    double t0 = cb * a[1] - sb * a[2] + b[1], t1 = sb * a[1] + cb * a[2] + b[2];
    out[0] = a[0] + b[0];
    out[1] = t0;
    out[2] = t1;
}
