/*
 * eecmg_oracle.c -- plain FP64 CPU restatement of the Extrapolation Economy
 * Cascadic Multigrid method (EECMG) for image restoration, Chu, Yan & Li,
 * "A New Extrapolation Economy Cascadic Multigrid Method for Image
 * Restoration Problems".
 *
 * TEST INFRASTRUCTURE.  This file is the checker the CUDA library is
 * compared against.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header,
 * table or helper with the CUDA library and must never be called from the
 * product path.
 *
 * Style: every operator is written as its definition, one output value at a
 * time, in FP64, with no blocking, fusion or reordering beyond what the
 * definition states.  The only parallelism is an optional OpenMP split over
 * output rows (each output value is computed independently, and every inner
 * product is summed row by row and then over rows in row order, so the
 * result is bitwise the same for any thread count).
 *
 * Conventions: an image of h rows and w columns is stored row-major,
 * x[i*w + j], 0-based.  A PSF K has kh rows and kw columns (both odd) and is
 * centred: K(p, q) = K[(p + ry)*kw + (q + rx)], ry = kh/2, rx = kw/2.
 *
 * Readings of passages the paper leaves open (each marked "Reading" below):
 * zero boundary for H; restriction = injection of even 0-based pixels;
 * R_l^* is the adjoint under the RMS inner product of Eq. 10; "CG" = CGLS
 * and "MR" = MR-II; Pi's value at cell centres; index clamping at the
 * right/bottom edge; the local-fit pseudo-inverse; the explicit PM step with
 * central-difference gradient and zero-flux boundary.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------ */
/* threads                                                              */
/* ------------------------------------------------------------------ */

OR_API void or_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

OR_API int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* vectors and the inner product                                        */
/* ------------------------------------------------------------------ */

/* <x, y> = sum_i x_i y_i, summed within each row, then over rows in order. */
OR_API double or_dot(const double *x, const double *y, int h, int w)
{
    double *row = (double *)malloc(sizeof(double) * (size_t)(h > 0 ? h : 1));
    int i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < h; ++i) {
        double s = 0.0;
        for (int j = 0; j < w; ++j)
            s += x[(size_t)i * w + j] * y[(size_t)i * w + j];
        row[i] = s;
    }
    double t = 0.0;
    for (i = 0; i < h; ++i)
        t += row[i];
    free(row);
    return t;
}

/* RMS norm of Eq. 10: ||v|| = ( (1/m) sum v_i^2 )^(1/2). */
OR_API double or_rms(const double *x, int h, int w)
{
    if (h * w == 0)
        return 0.0;
    return sqrt(or_dot(x, x, h, w) / ((double)h * (double)w));
}

static double *vec_new(size_t n)
{
    double *p = (double *)calloc(n ? n : 1, sizeof(double));
    return p;
}

/* The two stopping rules of the level smoothers (see or_mr2). */
static int level_done(const double *r, int h, int w, double stop_tol, double conv_lim)
{
    if (stop_tol > 0.0 && or_rms(r, h, w) <= stop_tol)
        return 1;
    if (conv_lim > 0.0 && sqrt(or_dot(r, r, h, w)) <= conv_lim)
        return 1;
    return 0;
}

/* ------------------------------------------------------------------ */
/* level sizes and restriction (Section 2, Eqs. 12-13)                  */
/* ------------------------------------------------------------------ */

/*
 * Nested grids G_1 c ... c G_L (Section 2): the next coarser side is
 * (n + 1)/2 for odd n and n/2 for even n, i.e. ceil(n/2), applied to each
 * side separately.  hs[0], ws[0] is the coarsest level G_1.
 */
OR_API void or_level_sizes(int h, int w, int L, int *hs, int *ws)
{
    hs[L - 1] = h;
    ws[L - 1] = w;
    for (int l = L - 1; l > 0; --l) {
        hs[l - 1] = (hs[l] + 1) / 2;
        ws[l - 1] = (ws[l] + 1) / 2;
    }
}

/*
 * Restriction R_l of Eqs. 12-13: the coarse value k is the fine value
 * 2k - 1 (1-based).  Reading: applied per dimension of the image, i.e. in
 * 0-based indices g_l(a, b) = g_{l+1}(2a, 2b).
 */
OR_API void or_restrict(const double *fine, int hf, int wf, double *coarse, int hc, int wc)
{
    (void)hf;
    for (int a = 0; a < hc; ++a)
        for (int b = 0; b < wc; ++b)
            coarse[(size_t)a * wc + b] = fine[(size_t)(2 * a) * wf + 2 * b];
}

/* ------------------------------------------------------------------ */
/* the blur operator H and its transpose (Eqs. 1-3, 7, 9)               */
/* ------------------------------------------------------------------ */

/*
 * y = H x: two-dimensional convolution with the PSF, Eq. 1 discretised as
 * Eq. 7.  The paper's H is block Toeplitz, so x is taken as zero outside
 * the image (no periodic or reflexive extension):
 *   y(i, j) = sum_{p, q} K(p, q) x(i - p, j - q).
 */
OR_API void or_apply_H(const double *K, int kh, int kw, const double *x, int h, int w, double *y)
{
    const int ry = kh / 2, rx = kw / 2;
    int i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < h; ++i) {
        for (int j = 0; j < w; ++j) {
            double s = 0.0;
            for (int p = -ry; p <= ry; ++p) {
                const int ii = i - p;
                if (ii < 0 || ii >= h)
                    continue;
                for (int q = -rx; q <= rx; ++q) {
                    const int jj = j - q;
                    if (jj < 0 || jj >= w)
                        continue;
                    s += K[(size_t)(p + ry) * kw + (q + rx)] * x[(size_t)ii * w + jj];
                }
            }
            y[(size_t)i * w + j] = s;
        }
    }
}

/*
 * y = H^T x: the transpose of the zero-boundary convolution is the
 * zero-boundary correlation y(i, j) = sum_{p, q} K(p, q) x(i + p, j + q).
 */
OR_API void or_apply_HT(const double *K, int kh, int kw, const double *x, int h, int w, double *y)
{
    const int ry = kh / 2, rx = kw / 2;
    int i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < h; ++i) {
        for (int j = 0; j < w; ++j) {
            double s = 0.0;
            for (int p = -ry; p <= ry; ++p) {
                const int ii = i + p;
                if (ii < 0 || ii >= h)
                    continue;
                for (int q = -rx; q <= rx; ++q) {
                    const int jj = j + q;
                    if (jj < 0 || jj >= w)
                        continue;
                    s += K[(size_t)(p + ry) * kw + (q + rx)] * x[(size_t)ii * w + jj];
                }
            }
            y[(size_t)i * w + j] = s;
        }
    }
}

/* ------------------------------------------------------------------ */
/* coarse operators H_l = R_l H_{l+1} R_l^* (Eq. 14)                    */
/* ------------------------------------------------------------------ */

/*
 * Eq. 14 with R_l the injection above and R_l^* its adjoint.  Reading: the
 * adjoint is taken under the inner product that induces the RMS norm of
 * Eq. 10, <x, y>_l = (1/N_l) sum x y, which gives R_l^* = rho * (zero-fill
 * upsampling), rho = N_{l+1} / N_l.  Writing the product out, the coarse
 * operator is again a zero-boundary convolution, with PSF
 *   K_l(p, q) = rho * K_{l+1}(2p, 2q),   |p| <= ry/2, |q| <= rx/2.
 * Returns the coarse PSF sizes in *kch, *kcw.
 */
OR_API void or_coarse_psf(const double *K, int kh, int kw, double rho, double *Kc, int *kch, int *kcw)
{
    const int ry = kh / 2, rx = kw / 2;
    const int cy = ry / 2, cx = rx / 2;
    const int ch = 2 * cy + 1, cw = 2 * cx + 1;
    for (int p = -cy; p <= cy; ++p)
        for (int q = -cx; q <= cx; ++q)
            Kc[(size_t)(p + cy) * cw + (q + cx)] = rho * K[(size_t)(2 * p + ry) * kw + (2 * q + rx)];
    *kch = ch;
    *kcw = cw;
}

/* ------------------------------------------------------------------ */
/* the economy iteration schedule m_l (Section 2)                        */
/* ------------------------------------------------------------------ */

/*
 * m_l = [ m_0 (L - L_0)^2 beta^(L-l) ]              for l > L_0,
 * m_l = [ m_*^(1/2) (L - (2 - eps_0) l) h_l^(-2) ]  for l <= L_0,
 * with L_0 = L/2, m_0 = 1, beta = 4, m_* = 1, eps_0 = 1/2, h_l = 2^(1-l),
 * and [t] the smallest positive integer not less than t.  Reading: L_0 is
 * the real number L/2 (not rounded).  m[0] is the coarsest level.
 * Every quantity is a multiple of 1/4 times a power of 4: exact in FP64.
 */
OR_API void or_schedule(int L, int *m)
{
    const double L0 = 0.5 * L;
    for (int l = 1; l <= L; ++l) {
        double t;
        if ((double)l > L0)
            t = (L - L0) * (L - L0) * pow(4.0, (double)(L - l));
        else
            t = (L - 1.5 * l) * pow(4.0, (double)(l - 1));
        int v = (int)ceil(t);
        m[l - 1] = v < 1 ? 1 : v;
    }
}

/* ------------------------------------------------------------------ */
/* the level smoothers C_l^m (Section 2): MR-II and CGLS                */
/* ------------------------------------------------------------------ */

/*
 * Reading of "MR" (Section 2): MR-II, the minimal-residual method whose
 * k-th iterate minimises ||g - H u|| over u_0 + span{H r_0, ..., H^k r_0}
 * (H symmetric).  Directions p_j with images q_j = H p_j kept mutually
 * orthogonal by a three-term recurrence:
 *   p_1 = H r_0,  q_1 = H p_1;
 *   z = H q_k,  b1 = <z, q_k>/<q_k, q_k>,  b2 = <z, q_{k-1}>/<q_{k-1}, q_{k-1}>,
 *   q_{k+1} = z - b1 q_k - b2 q_{k-1},   p_{k+1} = q_k - b1 p_k - b2 p_{k-1};
 *   a = <r, q_{k+1}>/<q_{k+1}, q_{k+1}>,  u += a p_{k+1},  r -= a q_{k+1}.
 * Breakdown (<q, q> not positive or not finite) ends the level with the
 * current iterate.  Two rules are checked before every iteration:
 *   discrepancy (Section 2; stop_tol > 0): stop if ||r||_RMS <= stop_tol;
 *   convergence (conv_tol > 0): stop if ||r|| <= conv_tol * ||g||.
 * Reading of the convergence rule: once the residual is zero the exact
 * method takes no further step (a = 0), so its remaining iterations leave u
 * unchanged; in floating point they would instead follow rounding noise
 * (the p_k recurrence drifts away from H^{-1} q_k and the iterate grows
 * without bound while the recursive residual stays tiny).  A level whose
 * residual has reached conv_tol relative to its data therefore ends there,
 * as an exact breakdown would.
 * u holds u_0 on entry and the result on exit.  res_rms (may be NULL)
 * receives ||g - H u||_RMS of the returned iterate.  Returns the number of
 * iterations taken.
 */
OR_API int or_mr2(const double *K, int kh, int kw, const double *g, int h, int w, double *u,
                  int m, double stop_tol, double conv_tol, double *res_rms)
{
    const size_t N = (size_t)h * w;
    double *r = vec_new(N), *p = vec_new(N), *q = vec_new(N);
    double *pp = vec_new(N), *qp = vec_new(N), *z = vec_new(N);
    double *pn = vec_new(N), *qn = vec_new(N);
    int k = 0;

    const double conv_lim = conv_tol > 0.0 ? conv_tol * sqrt(or_dot(g, g, h, w)) : 0.0;
    or_apply_H(K, kh, kw, u, h, w, r);
    for (size_t i = 0; i < N; ++i)
        r[i] = g[i] - r[i];

    if (m > 0 && !level_done(r, h, w, stop_tol, conv_lim)) {
        or_apply_H(K, kh, kw, r, h, w, p);
        or_apply_H(K, kh, kw, p, h, w, q);
        double qq = or_dot(q, q, h, w);
        if (qq > 0.0 && isfinite(qq)) {
            double a = or_dot(r, q, h, w) / qq;
            for (size_t i = 0; i < N; ++i) {
                u[i] += a * p[i];
                r[i] -= a * q[i];
            }
            k = 1;
            double qqp = 0.0;
            while (k < m) {
                if (level_done(r, h, w, stop_tol, conv_lim))
                    break;
                or_apply_H(K, kh, kw, q, h, w, z);
                double b1 = or_dot(z, q, h, w) / qq;
                double b2 = (k >= 2) ? or_dot(z, qp, h, w) / qqp : 0.0;
                for (size_t i = 0; i < N; ++i) {
                    qn[i] = z[i] - b1 * q[i] - b2 * qp[i];
                    pn[i] = q[i] - b1 * p[i] - b2 * pp[i];
                }
                double qqn = or_dot(qn, qn, h, w);
                if (!(qqn > 0.0) || !isfinite(qqn))
                    break;
                a = or_dot(r, qn, h, w) / qqn;
                for (size_t i = 0; i < N; ++i) {
                    u[i] += a * pn[i];
                    r[i] -= a * qn[i];
                }
                /* rotate: (p_{k-1}, q_{k-1}) <- (p_k, q_k) <- (p_{k+1}, q_{k+1}) */
                double *t;
                t = pp; pp = p; p = pn; pn = t;
                t = qp; qp = q; q = qn; qn = t;
                qqp = qq;
                qq = qqn;
                ++k;
            }
        }
    }
    if (res_rms)
        *res_rms = or_rms(r, h, w);
    free(r); free(p); free(q); free(pp); free(qp); free(z); free(pn); free(qn);
    return k;
}

/*
 * Reading of "CG" (Section 2): CGLS, conjugate gradients on the normal
 * equations H^T H u = H^T g, which minimises ||g - H u|| over
 * u_0 + span{H^T r_0, ..., (H^T H)^(k-1) H^T r_0} and needs no symmetry:
 *   s = H^T r, p = s, gamma = <s, s>;
 *   q = H p,  a = gamma/<q, q>,  u += a p,  r -= a q,
 *   s = H^T r,  gamma' = <s, s>,  p = s + (gamma'/gamma) p.
 * Same conventions and stopping rules as or_mr2.
 */
OR_API int or_cgls(const double *K, int kh, int kw, const double *g, int h, int w, double *u,
                   int m, double stop_tol, double conv_tol, double *res_rms)
{
    const size_t N = (size_t)h * w;
    double *r = vec_new(N), *s = vec_new(N), *p = vec_new(N), *q = vec_new(N);
    int k = 0;

    const double conv_lim = conv_tol > 0.0 ? conv_tol * sqrt(or_dot(g, g, h, w)) : 0.0;
    or_apply_H(K, kh, kw, u, h, w, r);
    for (size_t i = 0; i < N; ++i)
        r[i] = g[i] - r[i];
    or_apply_HT(K, kh, kw, r, h, w, s);
    memcpy(p, s, N * sizeof(double));
    double gamma = or_dot(s, s, h, w);
    while (k < m && gamma > 0.0 && isfinite(gamma)) {
        if (level_done(r, h, w, stop_tol, conv_lim))
            break;
        or_apply_H(K, kh, kw, p, h, w, q);
        double qq = or_dot(q, q, h, w);
        if (!(qq > 0.0) || !isfinite(qq))
            break;
        double a = gamma / qq;
        for (size_t i = 0; i < N; ++i) {
            u[i] += a * p[i];
            r[i] -= a * q[i];
        }
        ++k;
        or_apply_HT(K, kh, kw, r, h, w, s);
        double gn = or_dot(s, s, h, w);
        double beta = gn / gamma;
        for (size_t i = 0; i < N; ++i)
            p[i] = s[i] + beta * p[i];
        gamma = gn;
    }
    if (res_rms)
        *res_rms = or_rms(r, h, w);
    free(r); free(s); free(p); free(q);
    return k;
}

/* ------------------------------------------------------------------ */
/* prolongations (Section 3.1, 3.2)                                      */
/* ------------------------------------------------------------------ */

static int clampi(int v, int hi) { return v > hi ? hi : v; }

/*
 * New extrapolation Pi_l (Section 3.2): values on the level-(l-1) grid from
 * the final iterates u1 = u^{l-1} (h1 x w1) and u2 = u^{l-2} (h2 x w2).
 * With d = u^{l-1}|_{G_{l-2}} - u^{l-2} on the level-(l-2) nodes
 * (d(A, B) = u1(2A, 2B) - u2(A, B)), the printed cases are
 *   coarse node:   (5 u^{l-1} - u^{l-2}) / 4  =  u^{l-1} + d / 4,
 *   edge midpoint: u^{l-1} + (d_a + d_b) / 8,
 * i.e. u^{l-1} + (1/4) * (linear interpolant of d).  Reading: the cell
 * centre, not printed, is u^{l-1} + (1/16) * (sum of the four corner d),
 * the same rule; a level-(l-2) index past the last node is clamped to it.
 */
OR_API void or_extrapolate(const double *u1, int h1, int w1, const double *u2, int h2, int w2,
                           double *out)
{
    for (int a = 0; a < h1; ++a) {
        const int A0 = a / 2;
        const int A1 = (a & 1) ? clampi(A0 + 1, h2 - 1) : A0;
        for (int b = 0; b < w1; ++b) {
            const int B0 = b / 2;
            const int B1 = (b & 1) ? clampi(B0 + 1, w2 - 1) : B0;
            const int As[2] = {A0, A1}, Bs[2] = {B0, B1};
            double dsum = 0.0;
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) {
                    const int A = As[i], B = Bs[j];
                    dsum += u1[(size_t)(2 * A) * w1 + 2 * B] - u2[(size_t)A * w2 + B];
                }
            out[(size_t)a * w1 + b] = u1[(size_t)a * w1 + b] + 0.25 * (0.25 * dsum);
        }
    }
}

/*
 * Quadratic interpolation P_l (Section 3.2): on each level-(l-2) cell the
 * level-(l-1) triplet at indices 2A, 2A+1, 2A+2 carries a quadratic; the
 * level-l points of that cell sit at offsets 0, 1/4, 1/2, 3/4 of it, where
 * three-point Lagrange interpolation has weights
 *   t = 0: (1, 0, 0),  t = 1/4: (3/8, 3/4, -1/8),
 *   t = 1/2: (0, 1, 0),  t = 3/4: (-1/8, 3/4, 3/8).
 * In two dimensions the rule is applied along rows and along columns (a
 * tensor product; the two orders give the same value).  Reading: a
 * level-(l-1) index past the last node is clamped to it.
 * ut is h1 x w1 (level l-1); out is h x w (level l).
 */
static const double QW[4][3] = {
    {1.0, 0.0, 0.0}, {0.375, 0.75, -0.125}, {0.0, 1.0, 0.0}, {-0.125, 0.75, 0.375}};

OR_API void or_quadratic(const double *ut, int h1, int w1, double *out, int h, int w)
{
    int y;
#pragma omp parallel for schedule(static)
    for (y = 0; y < h; ++y) {
        const int A = y / 4, ty = y % 4;
        for (int x = 0; x < w; ++x) {
            const int B = x / 4, tx = x % 4;
            double s = 0.0;
            for (int i = 0; i < 3; ++i) {
                const int a = clampi(2 * A + i, h1 - 1);
                for (int j = 0; j < 3; ++j) {
                    const int b = clampi(2 * B + j, w1 - 1);
                    s += QW[ty][i] * QW[tx][j] * ut[(size_t)a * w1 + b];
                }
            }
            out[(size_t)y * w + x] = s;
        }
    }
}

/*
 * Linear prolongation L_l, Eq. 15 (Algorithm 1, IECMG-L).  In 0-based
 * indices: fine (2a, 2b) copies coarse (a, b); (2a, 2b+1) averages the two
 * horizontal neighbours; (2a+1, 2b) the two vertical ones; (2a+1, 2b+1)
 * averages the diagonal pair (a, b), (a+1, b+1).  Reading: indices past the
 * last coarse node are clamped to it.
 */
OR_API void or_linear(const double *uc, int hc, int wc, double *out, int h, int w)
{
    for (int y = 0; y < h; ++y) {
        const int a = y / 2, a1 = clampi(a + 1, hc - 1);
        for (int x = 0; x < w; ++x) {
            const int b = x / 2, b1 = clampi(b + 1, wc - 1);
            double v;
            if (!(y & 1) && !(x & 1))
                v = uc[(size_t)a * wc + b];
            else if (!(y & 1))
                v = 0.5 * (uc[(size_t)a * wc + b] + uc[(size_t)a * wc + b1]);
            else if (!(x & 1))
                v = 0.5 * (uc[(size_t)a * wc + b] + uc[(size_t)a1 * wc + b]);
            else
                v = 0.5 * (uc[(size_t)a * wc + b] + uc[(size_t)a1 * wc + b1]);
            out[(size_t)y * w + x] = v;
        }
    }
}

/* ------------------------------------------------------------------ */
/* local smoothing S_l (Section 3.3, Eqs. 18-19)                        */
/* ------------------------------------------------------------------ */

/*
 * For each pixel, the weighted least-squares plane fit of Eq. 19 over its
 * 3 x 3 neighbourhood with the weights of Eq. 18,
 *   w(s, t) = exp(-(scale * (u(i, j) - u(i+s, j+t)))^2),
 * and the output is the fitted constant a0.  Readings: scale = 1 is the
 * literal weight on the [0, 255] grey scale; neighbours outside the image
 * are left out; the fit is solved in centred form (values
 * v = u(i+s, j+t) - u(i, j), weighted means sb, tb, vb, 2 x 2 moment matrix
 * C and cross vector c), slope = C^+ c with eigenvalues below 1e-6 * W
 * (W = sum of weights) treated as zero, and a0 = u + vb - slope . (sb, tb).
 * a0 is unique even when C is singular because the centre has weight 1.
 */
OR_API void or_smooth(const double *u, int h, int w, double scale, double *out)
{
    int i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < h; ++i) {
        for (int j = 0; j < w; ++j) {
            const double uc = u[(size_t)i * w + j];
            double ws[9], ss[9], ts[9], vs[9];
            int n = 0;
            for (int s = -1; s <= 1; ++s)
                for (int t = -1; t <= 1; ++t) {
                    const int ii = i + s, jj = j + t;
                    if (ii < 0 || ii >= h || jj < 0 || jj >= w)
                        continue;
                    const double v = u[(size_t)ii * w + jj] - uc;
                    const double e = scale * v;
                    ws[n] = exp(-e * e);
                    ss[n] = s;
                    ts[n] = t;
                    vs[n] = v;
                    ++n;
                }
            double W = 0, sb = 0, tb = 0, vb = 0;
            for (int k = 0; k < n; ++k) {
                W += ws[k];
                sb += ws[k] * ss[k];
                tb += ws[k] * ts[k];
                vb += ws[k] * vs[k];
            }
            sb /= W;
            tb /= W;
            vb /= W;
            double css = 0, cst = 0, ctt = 0, csv = 0, ctv = 0;
            for (int k = 0; k < n; ++k) {
                const double ds = ss[k] - sb, dt = ts[k] - tb, dv = vs[k] - vb;
                css += ws[k] * ds * ds;
                cst += ws[k] * ds * dt;
                ctt += ws[k] * dt * dt;
                csv += ws[k] * ds * dv;
                ctv += ws[k] * dt * dv;
            }
            /* slope = C^+ c through the eigen-decomposition of the 2 x 2 C */
            const double tr = 0.5 * (css + ctt);
            const double df = 0.5 * (css - ctt);
            const double rad = sqrt(df * df + cst * cst);
            const double l1 = tr + rad, l2 = tr - rad;
            const double thr = 1e-6 * W;
            double e1s, e1t;                 /* unit eigenvector of l1 */
            if (rad > 0.0) {
                /* (C - l2 I) has rank one with columns along the l1 eigenvector */
                const double a0 = css - l2, b0 = cst, c0 = ctt - l2;
                if (fabs(a0) >= fabs(c0)) {
                    const double nn = sqrt(a0 * a0 + b0 * b0);
                    e1s = a0 / nn;
                    e1t = b0 / nn;
                } else {
                    const double nn = sqrt(b0 * b0 + c0 * c0);
                    e1s = b0 / nn;
                    e1t = c0 / nn;
                }
            } else {
                e1s = 1.0;
                e1t = 0.0;
            }
            const double e2s = -e1t, e2t = e1s;
            double gs = 0.0, gt = 0.0;
            if (l1 > thr) {
                const double c1 = (e1s * csv + e1t * ctv) / l1;
                gs += c1 * e1s;
                gt += c1 * e1t;
            }
            if (l2 > thr) {
                const double c2 = (e2s * csv + e2t * ctv) / l2;
                gs += c2 * e2s;
                gt += c2 * e2t;
            }
            out[(size_t)i * w + j] = uc + vb - (gs * sb + gt * tb);
        }
    }
}

/* ------------------------------------------------------------------ */
/* edge-preserving denoising D_l (Section 4, Eqs. 20-26)                */
/* ------------------------------------------------------------------ */

/*
 * One explicit step of the Perona-Malik equation (Eqs. 20-21) in the form
 * of Eqs. 23-24:
 *   u'(i, j) = u(i, j) + tau * sum_{(k,l) in Q(i,j)} (c(k,l) + c(i,j))/2
 *                                                   * (u(k, l) - u(i, j)),
 * with c = 1 / (1 + (|grad u| / k)^2) (Eq. 21) and Q the four neighbours.
 * Readings: |grad u| by central differences, an out-of-image neighbour
 * replaced by the centre value; neighbours outside the image contribute no
 * flux (terms omitted); one step per call.
 */
OR_API void or_denoise(const double *u, int h, int w, double tau, double kpm, double *out)
{
    const size_t N = (size_t)h * w;
    double *c = vec_new(N);
    int i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < h; ++i) {
        for (int j = 0; j < w; ++j) {
            const double uc = u[(size_t)i * w + j];
            const double ue = (j + 1 < w) ? u[(size_t)i * w + j + 1] : uc;
            const double uw = (j - 1 >= 0) ? u[(size_t)i * w + j - 1] : uc;
            const double us = (i + 1 < h) ? u[(size_t)(i + 1) * w + j] : uc;
            const double un = (i - 1 >= 0) ? u[(size_t)(i - 1) * w + j] : uc;
            const double gx = 0.5 * (ue - uw), gy = 0.5 * (us - un);
            c[(size_t)i * w + j] = 1.0 / (1.0 + (gx * gx + gy * gy) / (kpm * kpm));
        }
    }
#pragma omp parallel for schedule(static)
    for (i = 0; i < h; ++i) {
        for (int j = 0; j < w; ++j) {
            const size_t o = (size_t)i * w + j;
            const double uc = u[o], cc = c[o];
            double f = 0.0;
            if (i + 1 < h) f += 0.5 * (c[o + w] + cc) * (u[o + w] - uc);
            if (i - 1 >= 0) f += 0.5 * (c[o - w] + cc) * (u[o - w] - uc);
            if (j + 1 < w) f += 0.5 * (c[o + 1] + cc) * (u[o + 1] - uc);
            if (j - 1 >= 0) f += 0.5 * (c[o - 1] + cc) * (u[o - 1] - uc);
            out[o] = uc + tau * f;
        }
    }
    free(c);
}

/* ------------------------------------------------------------------ */
/* the cascade (Algorithm 2, EECMG; Algorithm 1, IECMG)                  */
/* ------------------------------------------------------------------ */

enum { OR_MR2 = 0, OR_CGLS = 1 };
enum { OR_GALERKIN_RMS = 0, OR_GALERKIN_RENORM = 1 };
enum { OR_EECMG = 0, OR_IECMG_P = 1, OR_IECMG_L = 2 };

typedef struct {
    int smoother;         /* OR_MR2 or OR_CGLS                                */
    int coarse_op;        /* OR_GALERKIN_RMS or OR_GALERKIN_RENORM            */
    int prolong;          /* OR_EECMG (Alg. 2) or OR_IECMG_P / _L (Alg. 1)    */
    int stop;             /* 0: exactly m_l iterations; 1: discrepancy rule   */
    double c;             /* discrepancy constant c > 1                        */
    double delta;         /* noise level delta = ||e||_RMS                     */
    int diffusion_steps;  /* explicit PM steps per prolonged level            */
    double s_scale;       /* scale of the S_l weight argument                  */
    double conv_tol;      /* convergence stop ||r|| <= conv_tol ||g_l|| (0: off) */
} or_options;

static int psf_is_zero(const double *K, int n)
{
    for (int i = 0; i < n; ++i)
        if (K[i] != 0.0)
            return 0;
    return 1;
}

static void solve_level(const or_options *o, const double *K, int kh, int kw, const double *g,
                        int h, int w, double *u, int m, int *it, double *res)
{
    const double tol = o->stop == 1 ? o->c * o->delta : 0.0;
    if (o->smoother == OR_CGLS)
        *it = or_cgls(K, kh, kw, g, h, w, u, m, tol, o->conv_tol, res);
    else
        *it = or_mr2(K, kh, kw, g, h, w, u, m, tol, o->conv_tol, res);
}

/*
 * EECMG, Algorithm 2, with the operators above.
 *   Sizes and data pyramid: Section 2, Eqs. 12-13.  Operators: Eq. 14.
 *   Step 1: u_l = C_l^{m_l} 0 for the two coarsest levels.
 *   Step 2: for each finer level l: u~' = Pi(u_{l-1}, u_{l-2}) on G_{l-1},
 *           u~ = P(u~'), then S, then D, then u_l = C_l^{m_l} u~.
 *   Step 3: output u_L.
 * Readings: the loop of Step 2 runs so that it produces levels 3..L
 * (L >= 3 for any prolonged level; L = 1 or 2 solve from zero only); Pi
 * takes the final iterates of the two previous levels; S and D act only on
 * prolonged levels.  With o->prolong = OR_IECMG_P / OR_IECMG_L the cascade
 * is Algorithm 1 instead: only the coarsest level starts from zero, and
 * every finer level starts from P(u_{l-1}) (quadratic, no extrapolation) or
 * L(u_{l-1}) (Eq. 15).
 * iters: per-level m_l, coarsest first, or NULL for the schedule above.
 * it_done, res_rms (may be NULL): per-level iterations and final ||r||_RMS.
 * Returns 0, or -1 on invalid arguments.
 */
OR_API int or_cascade(const double *g, int h, int w, int L, const double *psf, int kh, int kw,
                      double tau, double kpm, const int *iters, const or_options *o,
                      double *u_out, int *it_done, double *res_rms)
{
    if (L < 1 || h < 1 || w < 1 || !(kh & 1) || !(kw & 1))
        return -1;
    int *hs = (int *)malloc(sizeof(int) * L), *ws = (int *)malloc(sizeof(int) * L);
    int *m = (int *)malloc(sizeof(int) * L);
    or_level_sizes(h, w, L, hs, ws);
    if (iters)
        memcpy(m, iters, sizeof(int) * L);
    else
        or_schedule(L, m);

    double **gl = (double **)calloc(L, sizeof(double *));
    double **ul = (double **)calloc(L, sizeof(double *));
    double **Kl = (double **)calloc(L, sizeof(double *));
    int *khl = (int *)malloc(sizeof(int) * L), *kwl = (int *)malloc(sizeof(int) * L);

    for (int l = 0; l < L; ++l) {
        gl[l] = vec_new((size_t)hs[l] * ws[l]);
        ul[l] = vec_new((size_t)hs[l] * ws[l]);
    }
    memcpy(gl[L - 1], g, sizeof(double) * (size_t)h * w);
    for (int l = L - 1; l > 0; --l)
        or_restrict(gl[l], hs[l], ws[l], gl[l - 1], hs[l - 1], ws[l - 1]);

    Kl[L - 1] = vec_new((size_t)kh * kw);
    memcpy(Kl[L - 1], psf, sizeof(double) * (size_t)kh * kw);
    khl[L - 1] = kh;
    kwl[L - 1] = kw;
    double sum_fine = 0.0;
    for (int i = 0; i < kh * kw; ++i)
        sum_fine += psf[i];
    for (int l = L - 1; l > 0; --l) {
        const double rho = ((double)hs[l] * ws[l]) / ((double)hs[l - 1] * ws[l - 1]);
        const int ch = 2 * (khl[l] / 2 / 2) + 1, cw = 2 * (kwl[l] / 2 / 2) + 1;
        Kl[l - 1] = vec_new((size_t)ch * cw);
        or_coarse_psf(Kl[l], khl[l], kwl[l], rho, Kl[l - 1], &khl[l - 1], &kwl[l - 1]);
        if (o->coarse_op == OR_GALERKIN_RENORM) {
            /* Reading (flag): rescale each coarse PSF to the fine PSF's sum */
            double s = 0.0;
            const int n = khl[l - 1] * kwl[l - 1];
            for (int i = 0; i < n; ++i)
                s += Kl[l - 1][i];
            if (s != 0.0 && !psf_is_zero(Kl[l - 1], n))
                for (int i = 0; i < n; ++i)
                    Kl[l - 1][i] *= sum_fine / s;
        }
    }

    const int nzero = (o->prolong == OR_EECMG) ? 2 : 1;
    for (int l = 0; l < L; ++l) {
        const size_t N = (size_t)hs[l] * ws[l];
        int it = 0;
        double res = 0.0;
        if (l >= nzero) {
            double *ut = vec_new(N), *tmp = vec_new(N);
            if (o->prolong == OR_EECMG) {
                double *ue = vec_new((size_t)hs[l - 1] * ws[l - 1]);
                or_extrapolate(ul[l - 1], hs[l - 1], ws[l - 1], ul[l - 2], hs[l - 2], ws[l - 2], ue);
                or_quadratic(ue, hs[l - 1], ws[l - 1], ut, hs[l], ws[l]);
                free(ue);
            } else if (o->prolong == OR_IECMG_P) {
                or_quadratic(ul[l - 1], hs[l - 1], ws[l - 1], ut, hs[l], ws[l]);
            } else {
                or_linear(ul[l - 1], hs[l - 1], ws[l - 1], ut, hs[l], ws[l]);
            }
            or_smooth(ut, hs[l], ws[l], o->s_scale, tmp);
            for (int d = 0; d < o->diffusion_steps; ++d) {
                or_denoise(tmp, hs[l], ws[l], tau, kpm, ut);
                memcpy(tmp, ut, sizeof(double) * N);
            }
            memcpy(ul[l], tmp, sizeof(double) * N);
            free(ut);
            free(tmp);
        }
        solve_level(o, Kl[l], khl[l], kwl[l], gl[l], hs[l], ws[l], ul[l], m[l], &it, &res);
        if (it_done)
            it_done[l] = it;
        if (res_rms)
            res_rms[l] = res;
    }
    memcpy(u_out, ul[L - 1], sizeof(double) * (size_t)h * w);

    for (int l = 0; l < L; ++l) {
        free(gl[l]);
        free(ul[l]);
        free(Kl[l]);
    }
    free(gl); free(ul); free(Kl); free(khl); free(kwl); free(hs); free(ws); free(m);
    return 0;
}

/* PSNR of Section 5: 20 log10(255 / ||u - u_hat||) with the RMS norm. */
OR_API double or_psnr(const double *u, const double *uh, int h, int w)
{
    const size_t N = (size_t)h * w;
    double s = 0.0;
    for (size_t i = 0; i < N; ++i) {
        const double d = u[i] - uh[i];
        s += d * d;
    }
    return 20.0 * log10(255.0 / sqrt(s / (double)N));
}

/* ------------------------------------------------------------------ */
/* volumes (Section 6: the method carried over to three dimensions)     */
/* ------------------------------------------------------------------ */

/*
 * The paper names 3-D problems as the next application of the method and
 * gives no 3-D formulas, so every operator below is the 2-D one above with
 * the third axis treated exactly like the other two.  A volume of d slices,
 * h rows and w columns is stored x[(k*h + i)*w + j]; a PSF has kd x kh x kw
 * entries (all odd), centred: K(o, p, q) = K[((o+rz)*kh + p+ry)*kw + q+rx].
 * Readings (each "Reading 3-D" below): restriction injects even 0-based
 * voxels; Eq. 14 with the RMS adjoint gives K_l(o,p,q) = rho K(2o,2p,2q),
 * rho = N_{l+1}/N_l; Pi adds 1/4 of the trilinear interpolant of the
 * level-(l-2) differences; P is the tensor product of the three-point
 * quadratic rule along all three axes; S fits a hyperplane over the 3x3x3
 * neighbourhood with the Eq. 18 weights (3x3 moment matrix, pseudo-inverse
 * through a Jacobi eigen-decomposition); D takes the six face neighbours;
 * the smoother is MR-II and the iteration cap is the 2-D schedule m_l.
 * Inner products sum along rows, then over the d*h rows in order, as or_dot.
 */

OR_API void or_level_sizes3(int d, int h, int w, int L, int *ds, int *hs, int *ws)
{
    ds[L - 1] = d;
    or_level_sizes(h, w, L, hs, ws);
    for (int l = L - 1; l > 0; --l)
        ds[l - 1] = (ds[l] + 1) / 2;
}

/* Reading 3-D: coarse (a, b, c) = fine (2a, 2b, 2c), 0-based. */
OR_API void or_restrict3(const double *fine, int df, int hf, int wf, double *coarse, int dc,
                         int hc, int wc)
{
    (void)df;
    for (int a = 0; a < dc; ++a)
        for (int b = 0; b < hc; ++b)
            for (int c = 0; c < wc; ++c)
                coarse[((size_t)a * hc + b) * wc + c] =
                    fine[((size_t)(2 * a) * hf + 2 * b) * wf + 2 * c];
}

/*
 * y = H x (sgn = -1: convolution, y(k,i,j) = sum K(o,p,q) x(k-o, i-p, j-q))
 * or y = H^T x (sgn = +1: correlation, x(k+o, i+p, j+q)), zero outside the
 * volume; the sum runs over o, then p, then q.
 */
static void apply3(const double *K, int kd, int kh, int kw, const double *x, int d, int h, int w,
                   double *y, int sgn)
{
    const int rz = kd / 2, ry = kh / 2, rx = kw / 2;
    int row;
#pragma omp parallel for schedule(static)
    for (row = 0; row < d * h; ++row) {
        const int k = row / h, i = row % h;
        for (int j = 0; j < w; ++j) {
            double s = 0.0;
            for (int o = -rz; o <= rz; ++o) {
                const int kk = k + sgn * o;
                if (kk < 0 || kk >= d)
                    continue;
                for (int p = -ry; p <= ry; ++p) {
                    const int ii = i + sgn * p;
                    if (ii < 0 || ii >= h)
                        continue;
                    for (int q = -rx; q <= rx; ++q) {
                        const int jj = j + sgn * q;
                        if (jj < 0 || jj >= w)
                            continue;
                        s += K[((size_t)(o + rz) * kh + (p + ry)) * kw + (q + rx)] *
                             x[((size_t)kk * h + ii) * w + jj];
                    }
                }
            }
            y[(size_t)row * w + j] = s;
        }
    }
}

OR_API void or_apply_H3(const double *K, int kd, int kh, int kw, const double *x, int d, int h,
                        int w, double *y)
{
    apply3(K, kd, kh, kw, x, d, h, w, y, -1);
}

OR_API void or_apply_HT3(const double *K, int kd, int kh, int kw, const double *x, int d, int h,
                         int w, double *y)
{
    apply3(K, kd, kh, kw, x, d, h, w, y, +1);
}

/* Reading 3-D of Eq. 14: K_l(o, p, q) = rho * K_{l+1}(2o, 2p, 2q). */
OR_API void or_coarse_psf3(const double *K, int kd, int kh, int kw, double rho, double *Kc,
                           int *kcd, int *kch, int *kcw)
{
    const int rz = kd / 2, ry = kh / 2, rx = kw / 2;
    const int cz = rz / 2, cy = ry / 2, cx = rx / 2;
    const int cd = 2 * cz + 1, ch = 2 * cy + 1, cw = 2 * cx + 1;
    for (int o = -cz; o <= cz; ++o)
        for (int p = -cy; p <= cy; ++p)
            for (int q = -cx; q <= cx; ++q)
                Kc[((size_t)(o + cz) * ch + (p + cy)) * cw + (q + cx)] =
                    rho * K[((size_t)(2 * o + rz) * kh + (2 * p + ry)) * kw + (2 * q + rx)];
    *kcd = cd;
    *kch = ch;
    *kcw = cw;
}

/*
 * MR-II on a volume: the same recurrence, stopping rules and breakdown test
 * as or_mr2, with H the 3-D convolution.  With d = 1 and kd = 1 every step
 * is the 2-D one, in the same order.
 */
OR_API int or_mr2_3(const double *K, int kd, int kh, int kw, const double *g, int d, int h, int w,
                    double *u, int m, double stop_tol, double conv_tol, double *res_rms)
{
    const int rows = d * h;
    const size_t N = (size_t)rows * w;
    double *r = vec_new(N), *p = vec_new(N), *q = vec_new(N);
    double *pp = vec_new(N), *qp = vec_new(N), *z = vec_new(N);
    double *pn = vec_new(N), *qn = vec_new(N);
    int k = 0;

    const double conv_lim = conv_tol > 0.0 ? conv_tol * sqrt(or_dot(g, g, rows, w)) : 0.0;
    or_apply_H3(K, kd, kh, kw, u, d, h, w, r);
    for (size_t i = 0; i < N; ++i)
        r[i] = g[i] - r[i];

    if (m > 0 && !level_done(r, rows, w, stop_tol, conv_lim)) {
        or_apply_H3(K, kd, kh, kw, r, d, h, w, p);
        or_apply_H3(K, kd, kh, kw, p, d, h, w, q);
        double qq = or_dot(q, q, rows, w);
        if (qq > 0.0 && isfinite(qq)) {
            double a = or_dot(r, q, rows, w) / qq;
            for (size_t i = 0; i < N; ++i) {
                u[i] += a * p[i];
                r[i] -= a * q[i];
            }
            k = 1;
            double qqp = 0.0;
            while (k < m) {
                if (level_done(r, rows, w, stop_tol, conv_lim))
                    break;
                or_apply_H3(K, kd, kh, kw, q, d, h, w, z);
                double b1 = or_dot(z, q, rows, w) / qq;
                double b2 = (k >= 2) ? or_dot(z, qp, rows, w) / qqp : 0.0;
                for (size_t i = 0; i < N; ++i) {
                    qn[i] = z[i] - b1 * q[i] - b2 * qp[i];
                    pn[i] = q[i] - b1 * p[i] - b2 * pp[i];
                }
                double qqn = or_dot(qn, qn, rows, w);
                if (!(qqn > 0.0) || !isfinite(qqn))
                    break;
                a = or_dot(r, qn, rows, w) / qqn;
                for (size_t i = 0; i < N; ++i) {
                    u[i] += a * pn[i];
                    r[i] -= a * qn[i];
                }
                double *t;
                t = pp; pp = p; p = pn; pn = t;
                t = qp; qp = q; q = qn; qn = t;
                qqp = qq;
                qq = qqn;
                ++k;
            }
        }
    }
    if (res_rms)
        *res_rms = or_rms(r, rows, w);
    free(r); free(p); free(q); free(pp); free(qp); free(z); free(pn); free(qn);
    return k;
}

/*
 * Pi on a volume (Reading 3-D): u^{l-1} + (1/4) * (trilinear interpolant of
 * d = u^{l-1}|_{G_{l-2}} - u^{l-2}), i.e. the mean of d over the eight
 * corners of the level-(l-2) cell (repeated where an index is even), with a
 * level-(l-2) index past the last node clamped to it.
 */
OR_API void or_extrapolate3(const double *u1, int d1, int h1, int w1, const double *u2, int d2,
                            int h2, int w2, double *out)
{
    for (int c = 0; c < d1; ++c) {
        const int C0 = c / 2, C1 = (c & 1) ? clampi(C0 + 1, d2 - 1) : C0;
        for (int a = 0; a < h1; ++a) {
            const int A0 = a / 2, A1 = (a & 1) ? clampi(A0 + 1, h2 - 1) : A0;
            for (int b = 0; b < w1; ++b) {
                const int B0 = b / 2, B1 = (b & 1) ? clampi(B0 + 1, w2 - 1) : B0;
                const int Cs[2] = {C0, C1}, As[2] = {A0, A1}, Bs[2] = {B0, B1};
                double dsum = 0.0;
                for (int x = 0; x < 2; ++x)
                    for (int i = 0; i < 2; ++i)
                        for (int j = 0; j < 2; ++j) {
                            const int Cc = Cs[x], A = As[i], B = Bs[j];
                            dsum += u1[((size_t)(2 * Cc) * h1 + 2 * A) * w1 + 2 * B] -
                                    u2[((size_t)Cc * h2 + A) * w2 + B];
                        }
                const size_t o = ((size_t)c * h1 + a) * w1 + b;
                out[o] = u1[o] + 0.25 * (0.125 * dsum);
            }
        }
    }
}

/* P on a volume (Reading 3-D): the QW rule along all three axes. */
OR_API void or_quadratic3(const double *ut, int d1, int h1, int w1, double *out, int d, int h,
                          int w)
{
    int row;
#pragma omp parallel for schedule(static)
    for (row = 0; row < d * h; ++row) {
        const int z = row / h, y = row % h;
        const int Z = z / 4, tz = z % 4, Y = y / 4, ty = y % 4;
        for (int x = 0; x < w; ++x) {
            const int X = x / 4, tx = x % 4;
            double s = 0.0;
            for (int k = 0; k < 3; ++k) {
                const int c = clampi(2 * Z + k, d1 - 1);
                for (int i = 0; i < 3; ++i) {
                    const int a = clampi(2 * Y + i, h1 - 1);
                    for (int j = 0; j < 3; ++j) {
                        const int b = clampi(2 * X + j, w1 - 1);
                        s += QW[tz][k] * QW[ty][i] * QW[tx][j] * ut[((size_t)c * h1 + a) * w1 + b];
                    }
                }
            }
            out[(size_t)row * w + x] = s;
        }
    }
}

/*
 * Eigen-decomposition of a symmetric 3 x 3 matrix by the cyclic Jacobi
 * method (Golub & Van Loan, Matrix Computations, Sec. 8.5): rotations in the
 * (0,1), (0,2), (1,2) planes, each zeroing its off-diagonal entry, repeated
 * until every off-diagonal entry is zero or negligible next to the
 * diagonal.  On return A's diagonal holds the eigenvalues and the columns of
 * V the unit eigenvectors.
 */
static void jacobi3(double A[3][3], double V[3][3])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            V[i][j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 64; ++sweep) {
        const double off = fabs(A[0][1]) + fabs(A[0][2]) + fabs(A[1][2]);
        const double dia = fabs(A[0][0]) + fabs(A[1][1]) + fabs(A[2][2]);
        if (off == 0.0 || off <= 1e-18 * dia)
            break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (A[p][q] == 0.0)
                    continue;
                /* t = tan(theta) of the smaller rotation zeroing A[p][q] */
                const double th = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 3; ++k) {        /* A <- A J (columns p, q) */
                    const double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {        /* A <- J^T A (rows p, q) */
                    const double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                A[p][q] = A[q][p] = 0.0;
                for (int k = 0; k < 3; ++k) {        /* V <- V J */
                    const double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
    }
}

/*
 * S on a volume (Reading 3-D): for each voxel, the weighted least-squares
 * fit of v = a0' + g . o over its 3 x 3 x 3 neighbourhood (offsets o, values
 * v = u(neighbour) - u(centre), weights exp(-(scale v)^2) of Eq. 18,
 * neighbours outside the volume left out), in centred form: weighted means
 * ob, vb, moment matrix C = sum w (o - ob)(o - ob)^T, cross vector
 * c = sum w (o - ob)(v - vb), slope = C^+ c with eigenvalues below 1e-6 W
 * treated as zero; the output is u + vb - slope . ob.
 */
OR_API void or_smooth3(const double *u, int d, int h, int w, double scale, double *out)
{
    int row;
#pragma omp parallel for schedule(static)
    for (row = 0; row < d * h; ++row) {
        const int k = row / h, i = row % h;
        for (int j = 0; j < w; ++j) {
            const double uc = u[((size_t)k * h + i) * w + j];
            double ws[27], os[27][3], vs[27];
            int n = 0;
            for (int r = -1; r <= 1; ++r)
                for (int s = -1; s <= 1; ++s)
                    for (int t = -1; t <= 1; ++t) {
                        const int kk = k + r, ii = i + s, jj = j + t;
                        if (kk < 0 || kk >= d || ii < 0 || ii >= h || jj < 0 || jj >= w)
                            continue;
                        const double v = u[((size_t)kk * h + ii) * w + jj] - uc;
                        const double e = scale * v;
                        ws[n] = exp(-e * e);
                        os[n][0] = r;
                        os[n][1] = s;
                        os[n][2] = t;
                        vs[n] = v;
                        ++n;
                    }
            double W = 0.0, ob[3] = {0, 0, 0}, vb = 0.0;
            for (int m = 0; m < n; ++m) {
                W += ws[m];
                for (int a = 0; a < 3; ++a)
                    ob[a] += ws[m] * os[m][a];
                vb += ws[m] * vs[m];
            }
            for (int a = 0; a < 3; ++a)
                ob[a] /= W;
            vb /= W;
            double C[3][3] = {{0}}, cv[3] = {0, 0, 0};
            for (int m = 0; m < n; ++m) {
                double dd[3];
                for (int a = 0; a < 3; ++a)
                    dd[a] = os[m][a] - ob[a];
                const double dv = vs[m] - vb;
                for (int a = 0; a < 3; ++a) {
                    for (int b = 0; b < 3; ++b)
                        C[a][b] += ws[m] * dd[a] * dd[b];
                    cv[a] += ws[m] * dd[a] * dv;
                }
            }
            double V[3][3];
            jacobi3(C, V);
            const double thr = 1e-6 * W;
            double g[3] = {0, 0, 0};
            for (int e = 0; e < 3; ++e) {
                const double lam = C[e][e];
                if (!(lam > thr))
                    continue;
                const double ce = (V[0][e] * cv[0] + V[1][e] * cv[1] + V[2][e] * cv[2]) / lam;
                for (int a = 0; a < 3; ++a)
                    g[a] += ce * V[a][e];
            }
            out[((size_t)k * h + i) * w + j] = uc + vb - (g[0] * ob[0] + g[1] * ob[1] + g[2] * ob[2]);
        }
    }
}

/*
 * D on a volume (Reading 3-D): one explicit Perona-Malik step with the six
 * face neighbours, |grad u| by central differences along the three axes
 * (an out-of-volume neighbour replaced by the centre), and no flux through
 * the volume's faces; the flux terms are summed slice-, row-, then column-
 * neighbours.
 */
OR_API void or_denoise3(const double *u, int d, int h, int w, double tau, double kpm, double *out)
{
    const size_t N = (size_t)d * h * w, sl = (size_t)h * w;
    double *c = vec_new(N);
    int row;
#pragma omp parallel for schedule(static)
    for (row = 0; row < d * h; ++row) {
        const int k = row / h, i = row % h;
        for (int j = 0; j < w; ++j) {
            const size_t o = (size_t)row * w + j;
            const double uc = u[o];
            const double ub = (k + 1 < d) ? u[o + sl] : uc, ua = (k - 1 >= 0) ? u[o - sl] : uc;
            const double us = (i + 1 < h) ? u[o + w] : uc, un = (i - 1 >= 0) ? u[o - w] : uc;
            const double ue = (j + 1 < w) ? u[o + 1] : uc, uw = (j - 1 >= 0) ? u[o - 1] : uc;
            const double gx = 0.5 * (ue - uw), gy = 0.5 * (us - un), gz = 0.5 * (ub - ua);
            c[o] = 1.0 / (1.0 + (gx * gx + gy * gy + gz * gz) / (kpm * kpm));
        }
    }
#pragma omp parallel for schedule(static)
    for (row = 0; row < d * h; ++row) {
        const int k = row / h, i = row % h;
        for (int j = 0; j < w; ++j) {
            const size_t o = (size_t)row * w + j;
            const double uc = u[o], cc = c[o];
            double f = 0.0;
            if (k + 1 < d) f += 0.5 * (c[o + sl] + cc) * (u[o + sl] - uc);
            if (k - 1 >= 0) f += 0.5 * (c[o - sl] + cc) * (u[o - sl] - uc);
            if (i + 1 < h) f += 0.5 * (c[o + w] + cc) * (u[o + w] - uc);
            if (i - 1 >= 0) f += 0.5 * (c[o - w] + cc) * (u[o - w] - uc);
            if (j + 1 < w) f += 0.5 * (c[o + 1] + cc) * (u[o + 1] - uc);
            if (j - 1 >= 0) f += 0.5 * (c[o - 1] + cc) * (u[o - 1] - uc);
            out[o] = uc + tau * f;
        }
    }
    free(c);
}

/*
 * EECMG (Algorithm 2) on a volume, the steps of or_cascade with the 3-D
 * operators above.  Only o->smoother = OR_MR2 and o->prolong = OR_EECMG are
 * defined here; coarse_op, stop, c, delta, diffusion_steps, s_scale and
 * conv_tol mean what they mean in 2-D.  Returns 0, or -1 on invalid
 * arguments.
 */
OR_API int or_cascade3(const double *g, int d, int h, int w, int L, const double *psf, int kd,
                       int kh, int kw, double tau, double kpm, const int *iters,
                       const or_options *o, double *u_out, int *it_done, double *res_rms)
{
    if (L < 1 || d < 1 || h < 1 || w < 1 || !(kd & 1) || !(kh & 1) || !(kw & 1) ||
        o->smoother != OR_MR2 || o->prolong != OR_EECMG)
        return -1;
    int *ds = (int *)malloc(sizeof(int) * L), *hs = (int *)malloc(sizeof(int) * L);
    int *ws = (int *)malloc(sizeof(int) * L), *m = (int *)malloc(sizeof(int) * L);
    or_level_sizes3(d, h, w, L, ds, hs, ws);
    if (iters)
        memcpy(m, iters, sizeof(int) * L);
    else
        or_schedule(L, m);

    double **gl = (double **)calloc(L, sizeof(double *));
    double **ul = (double **)calloc(L, sizeof(double *));
    double **Kl = (double **)calloc(L, sizeof(double *));
    int *kdl = (int *)malloc(sizeof(int) * L), *khl = (int *)malloc(sizeof(int) * L);
    int *kwl = (int *)malloc(sizeof(int) * L);
    size_t *Nl = (size_t *)malloc(sizeof(size_t) * L);

    for (int l = 0; l < L; ++l) {
        Nl[l] = (size_t)ds[l] * hs[l] * ws[l];
        gl[l] = vec_new(Nl[l]);
        ul[l] = vec_new(Nl[l]);
    }
    memcpy(gl[L - 1], g, sizeof(double) * Nl[L - 1]);
    for (int l = L - 1; l > 0; --l)
        or_restrict3(gl[l], ds[l], hs[l], ws[l], gl[l - 1], ds[l - 1], hs[l - 1], ws[l - 1]);

    Kl[L - 1] = vec_new((size_t)kd * kh * kw);
    memcpy(Kl[L - 1], psf, sizeof(double) * (size_t)kd * kh * kw);
    kdl[L - 1] = kd;
    khl[L - 1] = kh;
    kwl[L - 1] = kw;
    double sum_fine = 0.0;
    for (int i = 0; i < kd * kh * kw; ++i)
        sum_fine += psf[i];
    for (int l = L - 1; l > 0; --l) {
        const double rho = (double)Nl[l] / (double)Nl[l - 1];
        const int cd = 2 * (kdl[l] / 2 / 2) + 1, ch = 2 * (khl[l] / 2 / 2) + 1;
        const int cw = 2 * (kwl[l] / 2 / 2) + 1;
        Kl[l - 1] = vec_new((size_t)cd * ch * cw);
        or_coarse_psf3(Kl[l], kdl[l], khl[l], kwl[l], rho, Kl[l - 1], &kdl[l - 1], &khl[l - 1],
                       &kwl[l - 1]);
        if (o->coarse_op == OR_GALERKIN_RENORM) {
            double s = 0.0;
            const int n = kdl[l - 1] * khl[l - 1] * kwl[l - 1];
            for (int i = 0; i < n; ++i)
                s += Kl[l - 1][i];
            if (s != 0.0 && !psf_is_zero(Kl[l - 1], n))
                for (int i = 0; i < n; ++i)
                    Kl[l - 1][i] *= sum_fine / s;
        }
    }

    const double tol = o->stop == 1 ? o->c * o->delta : 0.0;
    for (int l = 0; l < L; ++l) {
        const size_t N = Nl[l];
        if (l >= 2) {
            double *ut = vec_new(N), *tmp = vec_new(N), *ue = vec_new(Nl[l - 1]);
            or_extrapolate3(ul[l - 1], ds[l - 1], hs[l - 1], ws[l - 1], ul[l - 2], ds[l - 2],
                            hs[l - 2], ws[l - 2], ue);
            or_quadratic3(ue, ds[l - 1], hs[l - 1], ws[l - 1], ut, ds[l], hs[l], ws[l]);
            or_smooth3(ut, ds[l], hs[l], ws[l], o->s_scale, tmp);
            for (int s = 0; s < o->diffusion_steps; ++s) {
                or_denoise3(tmp, ds[l], hs[l], ws[l], tau, kpm, ut);
                memcpy(tmp, ut, sizeof(double) * N);
            }
            memcpy(ul[l], tmp, sizeof(double) * N);
            free(ut);
            free(tmp);
            free(ue);
        }
        double res = 0.0;
        const int it = or_mr2_3(Kl[l], kdl[l], khl[l], kwl[l], gl[l], ds[l], hs[l], ws[l], ul[l],
                                m[l], tol, o->conv_tol, &res);
        if (it_done)
            it_done[l] = it;
        if (res_rms)
            res_rms[l] = res;
    }
    memcpy(u_out, ul[L - 1], sizeof(double) * Nl[L - 1]);

    for (int l = 0; l < L; ++l) {
        free(gl[l]);
        free(ul[l]);
        free(Kl[l]);
    }
    free(gl); free(ul); free(Kl); free(kdl); free(khl); free(kwl); free(Nl);
    free(ds); free(hs); free(ws); free(m);
    return 0;
}
