/*
 * kzk_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU restatement of the exponential-integrator / WENO5
 * scheme of Einkemmer, Ostermann & Residori (arXiv:2103.06080), used to check
 * the CUDA library.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark may load it; the product path never calls it.  It shares no
 * code, header, table or constant generator with the CUDA library.
 *
 * Everything is written for clarity, in the order and notation of the paper:
 *   - grid: periodic in retarded time tau (x, contiguous) and transverse y
 *     (Sec. 3.3, "periodic boundary conditions both in rho and theta");
 *   - linear operator  L = (1/4pi) d_tau^{-1} d_y^2 + A d_tau^2     (Eq. 2),
 *     diagonal in Fourier space with the regularised multiplier of Eq. 11;
 *   - nonlinear part   b(sigma,V) = (B(sigma)/2) d_tau V^2           (Eq. 3,
 *     homogeneous medium) discretised by WENO5 on the gradient form of Eq. 7;
 *   - time integrator  ExpRK22 in Fourier space                      (Eq. 11,
 *     Algorithm 2, STEP 1-4).
 * Readings of points the paper leaves open (all stated in the design notes):
 *   WENO5 = Jiang-Shu weights, p = 2, linear weights (1/10, 6/10, 3/10);
 *   flux splitting = global Lax-Friedrichs with alpha = B(sigma) * M, M fixed;
 *   physical wavenumbers k = 2 pi m / length;  at the tau-Nyquist column the
 *   odd diffraction term is dropped (z = -dsigma * A * k_N^2);  sigma-varying
 *   absorption A(sigma) = A * pA(sigma) enters b as (A(sigma) - A) d_tau^2 V,
 *   because the paper keeps only constant-coefficient linear terms in L and
 *   puts every variable-coefficient term into b (Eq. 2 / Eq. 3).
 *
 * Build: gcc -O2 -fno-fast-math -ffp-contract=off -shared -fPIC [-fopenmp]
 * The -fopenmp build parallelises the independent rows / columns only; the
 * arithmetic of every value is the same as in the sequential build.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t nx, ny;                       /* grid points in tau and y */
    double tau_min, tau_max, y_min, y_max;
    double B, A;                          /* nonlinearity, absorption (Eq. 0) */
    double diffraction;                   /* 1/(4 pi) in Eq. 0 */
    double reg_eps;                       /* epsilon of the regularised multiplier (Eq. 11) */
    double weno_eps;                      /* Jiang-Shu epsilon */
    double lf_umax;                       /* M: Lax-Friedrichs alpha = B(sigma) * M */
    double B_prof[4], A_prof[4];          /* p(s) = c0 + c1 s + c2 s^2 + c3 s^3 in sigma */
    int32_t has_profile;                  /* 0: B, A constant */
    double dt;                            /* dsigma */
    int32_t n_relax;                      /* relaxation processes (0, 1 or 2) */
    double relax_C[2], relax_theta[2];    /* strength C_r and relaxation time theta_r of each */
    /* random inhomogeneous medium (Algorithm 1); n_modes = 0: homogeneous */
    int32_t n_modes;
    const double *mode_klam;              /* |K_n| lambda */
    const double *mode_theta;             /* theta_n: angle between K_n and the sigma axis */
    const double *mode_phase;             /* phi_n */
    const double *mode_amp;               /* |U~(K_n)| / c0 */
    int32_t method;                       /* 0: ExpRK22 (Eq. 5); 1: exponential Euler (Sec. 3.2) */
} orc_params;

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Mixed-radix FFT for lengths that are not powers of two (the paper's grids   */
/* have 7 * 2^k points in tau and 1250 * 2^k = 2^(k+1) * 5^4 in y, Table 1).    */
/* Recursive Cooley-Tukey decimation in time: with p the smallest prime factor */
/* of n and m = n / p, the p interleaved subsequences x_{p j + r} are          */
/* transformed (length m) and combined as                                      */
/*     X_k = sum_r exp(sgn 2 pi i r k / n) Y_r[k mod m];                        */
/* a prime length is the direct sum.  Unnormalised.                            */
/* ------------------------------------------------------------------------ */
static void fft_mixed(const double *xr, const double *xi, int stride, int n, double sgn, double *yr, double *yi)
{
    if (n == 1) { yr[0] = xr[0]; yi[0] = xi[0]; return; }
    int p = 2;
    while (n % p) p++;
    if (p == n) {
        for (int k = 0; k < n; k++) {
            double sr = 0.0, si = 0.0;
            for (int j = 0; j < n; j++) {
                /* exp(sgn 2 pi i j k / n), argument reduced modulo n */
                double ang = sgn * 2.0 * M_PI * (double)((long long)j * k % n) / (double)n;
                double wr = cos(ang), wi = sin(ang);
                sr += xr[(size_t)j * stride] * wr - xi[(size_t)j * stride] * wi;
                si += xr[(size_t)j * stride] * wi + xi[(size_t)j * stride] * wr;
            }
            yr[k] = sr; yi[k] = si;
        }
        return;
    }
    const int m = n / p;
    double *tr = (double *)malloc(sizeof(double) * n), *ti = (double *)malloc(sizeof(double) * n);
    for (int r = 0; r < p; r++)
        fft_mixed(xr + (size_t)r * stride, xi + (size_t)r * stride, stride * p, m, sgn, tr + (size_t)r * m,
                  ti + (size_t)r * m);
    for (int k = 0; k < n; k++) {
        double sr = 0.0, si = 0.0;
        for (int r = 0; r < p; r++) {
            double ang = sgn * 2.0 * M_PI * (double)((long long)r * k % n) / (double)n;
            double wr = cos(ang), wi = sin(ang);
            double ar = tr[(size_t)r * m + k % m], ai = ti[(size_t)r * m + k % m];
            sr += ar * wr - ai * wi;
            si += ar * wi + ai * wr;
        }
        yr[k] = sr; yi[k] = si;
    }
    free(tr); free(ti);
}

/* ------------------------------------------------------------------------ */
/* Radix-2 FFT (textbook iterative Cooley-Tukey, bit reversal + butterflies).  */
/* Forward: X_k = sum_n x_n exp(-2 pi i k n / N).  Inverse includes 1/N.       */
/* Other lengths: the mixed-radix transform above.                             */
/* ------------------------------------------------------------------------ */
void orc_fft1d(double *re, double *im, int n, int inverse)
{
    if (n & (n - 1)) {
        double *yr = (double *)malloc(sizeof(double) * n), *yi = (double *)malloc(sizeof(double) * n);
        fft_mixed(re, im, 1, n, inverse ? 1.0 : -1.0, yr, yi);
        for (int i = 0; i < n; i++) {
            re[i] = inverse ? yr[i] / n : yr[i];
            im[i] = inverse ? yi[i] / n : yi[i];
        }
        free(yr); free(yi);
        return;
    }
    /* bit-reversal permutation */
    for (int i = 1, j = 0; i < n; i++) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = re[i]; re[i] = re[j]; re[j] = t;
            t = im[i]; im[i] = im[j]; im[j] = t;
        }
    }
    const double sgn = inverse ? 1.0 : -1.0;
    for (int len = 2; len <= n; len <<= 1) {
        int half = len >> 1;
        for (int k = 0; k < half; k++) {
            /* twiddle exp(sgn * 2 pi i k / len), evaluated directly */
            double ang = sgn * 2.0 * M_PI * (double)k / (double)len;
            double wr = cos(ang), wi = sin(ang);
            for (int s = 0; s < n; s += len) {
                int a = s + k, b = s + k + half;
                double tr = re[b] * wr - im[b] * wi;
                double ti = re[b] * wi + im[b] * wr;
                re[b] = re[a] - tr; im[b] = im[a] - ti;
                re[a] = re[a] + tr; im[a] = im[a] + ti;
            }
        }
    }
    if (inverse) {
        for (int i = 0; i < n; i++) { re[i] /= n; im[i] /= n; }
    }
}

/* 2-D transform of a [ny][nx] complex array: along tau (rows), then along y. */
void orc_fft2d(double *re, double *im, int nx, int ny, int inverse)
{
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++) orc_fft1d(re + (size_t)j * nx, im + (size_t)j * nx, nx, inverse);
    #pragma omp parallel
    {
        double *cr = (double *)malloc(sizeof(double) * ny);
        double *ci = (double *)malloc(sizeof(double) * ny);
        #pragma omp for schedule(static)
        for (int m = 0; m < nx; m++) {
            for (int j = 0; j < ny; j++) { cr[j] = re[(size_t)j * nx + m]; ci[j] = im[(size_t)j * nx + m]; }
            orc_fft1d(cr, ci, ny, inverse);
            for (int j = 0; j < ny; j++) { re[(size_t)j * nx + m] = cr[j]; im[(size_t)j * nx + m] = ci[j]; }
        }
        free(cr); free(ci);
    }
}

/* Signed FFT index: m for m < n/2, m - n above; n/2 (Nyquist) kept positive. */
static int signed_index(int m, int n) { return (m <= n / 2) ? m : m - n; }

/* ------------------------------------------------------------------------ */
/* phi-functions of Eq. 5 / Eq. 11:  E = e^z,  Phi1 = (e^z - 1)/z,            */
/* Phi2 = (e^z - 1 - z)/z^2.  Near z = 0 the quotients cancel, so there the    */
/* Taylor series  Phi1 = sum z^n/(n+1)!,  Phi2 = sum z^n/(n+2)!  is summed.     */
/* ------------------------------------------------------------------------ */
typedef struct { double re, im; } cpx;
static cpx c_mk(double r, double i) { cpx c = {r, i}; return c; }
static cpx c_add(cpx a, cpx b) { return c_mk(a.re + b.re, a.im + b.im); }
static cpx c_sub(cpx a, cpx b) { return c_mk(a.re - b.re, a.im - b.im); }
static cpx c_mul(cpx a, cpx b) { return c_mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
static cpx c_div(cpx a, cpx b)
{
    /* Smith's algorithm: avoids overflow of |b|^2 */
    if (fabs(b.re) >= fabs(b.im)) {
        double r = b.im / b.re, d = b.re + b.im * r;
        return c_mk((a.re + a.im * r) / d, (a.im - a.re * r) / d);
    } else {
        double r = b.re / b.im, d = b.re * r + b.im;
        return c_mk((a.re * r + a.im) / d, (a.im * r - a.re) / d);
    }
}

void orc_phi(double zr, double zi, double *out /* E re,im, Phi1 re,im, Phi2 re,im */)
{
    cpx z = c_mk(zr, zi);
    double az = hypot(zr, zi);
    /* E = e^x (cos y + i sin y) */
    double ex = exp(zr);
    cpx E = c_mk(ex * cos(zi), ex * sin(zi));
    cpx P1, P2;
    if (az < 0.25) {
        /* Taylor series, summed from the highest term (Horner form) */
        cpx s1 = c_mk(0.0, 0.0), s2 = c_mk(0.0, 0.0);
        const int NT = 30;
        for (int n = NT; n >= 0; n--) {
            /* s1 <- 1/(n+1)! + z * s1 ;  s2 <- 1/(n+2)! + z * s2 */
            double f1 = 1.0, f2 = 1.0;
            for (int q = 2; q <= n + 1; q++) f1 *= q;
            for (int q = 2; q <= n + 2; q++) f2 *= q;
            s1 = c_add(c_mk(1.0 / f1, 0.0), c_mul(z, s1));
            s2 = c_add(c_mk(1.0 / f2, 0.0), c_mul(z, s2));
        }
        P1 = s1; P2 = s2;
    } else {
        /* e^z - 1 without cancellation: expm1(x) cos y - 2 sin^2(y/2) + i e^x sin y */
        double sh = sin(0.5 * zi);
        cpx Em1 = c_mk(expm1(zr) * cos(zi) - 2.0 * sh * sh, ex * sin(zi));
        P1 = c_div(Em1, z);
        P2 = c_div(c_sub(P1, c_mk(1.0, 0.0)), z);   /* (e^z-1-z)/z^2 = (Phi1 - 1)/z */
    }
    out[0] = E.re; out[1] = E.im; out[2] = P1.re; out[3] = P1.im; out[4] = P2.re; out[5] = P2.im;
}

/* z_{jk} of Eq. 11 with physical wavenumbers; j: y index, m: tau index. */
static cpx z_of(const orc_params *p, int j, int m)
{
    double Lx = p->tau_max - p->tau_min, Ly = p->y_max - p->y_min;
    double kt = 2.0 * M_PI * signed_index(m, p->nx) / Lx;
    double ky = 2.0 * M_PI * signed_index(j, p->ny) / Ly;
    double absorb = -p->A * kt * kt;
    /* relaxation: C_r d_tau^2 (1 + theta_r d_tau)^-1 per process; with
     * d_tau -> i kt its multiplier is C_r (i kt)^2 / (1 + i theta_r kt) */
    cpx relax = c_mk(0.0, 0.0);
    for (int r = 0; r < p->n_relax; r++)
        relax = c_add(relax, c_div(c_mk(-p->relax_C[r] * kt * kt, 0.0), c_mk(1.0, p->relax_theta[r] * kt)));
    if (p->nx > 1 && 2 * m == p->nx) {
        /* tau-Nyquist: only the even parts (absorption, the real part of the
         * relaxation multiplier) survive */
        return c_mk(p->dt * (absorb + relax.re), 0.0);
    }
    /* -diffraction * ky^2 / (i kt + eps * diffraction) - A kt^2 ; 1/(4 pi) = diffraction */
    cpx den = c_mk(p->reg_eps * p->diffraction, kt);
    cpx q = c_div(c_mk(-p->diffraction * ky * ky, 0.0), den);
    return c_mk(p->dt * (q.re + absorb + relax.re), p->dt * (q.im + relax.im));
}

/* Full (unfolded) tables, each [ny][nx] complex as separate re/im arrays. */
void orc_tables(const orc_params *p, double *Er, double *Ei, double *P1r, double *P1i,
                double *P2r, double *P2i)
{
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < p->ny; j++)
        for (int m = 0; m < p->nx; m++) {
            cpx z = z_of(p, j, m);
            double o[6];
            orc_phi(z.re, z.im, o);
            size_t i = (size_t)j * p->nx + m;
            Er[i] = o[0]; Ei[i] = o[1]; P1r[i] = o[2]; P1i[i] = o[3]; P2r[i] = o[4]; P2i[i] = o[5];
        }
}

/* Profile p(sigma) = c0 + c1 sigma + c2 sigma^2 + c3 sigma^3 (Horner). */
static double profile(const double *c, double s) { return ((c[3] * s + c[2]) * s + c[1]) * s + c[0]; }
double orc_B_of(const orc_params *p, double s) { return p->has_profile ? p->B * profile(p->B_prof, s) : p->B; }
double orc_A_of(const orc_params *p, double s) { return p->has_profile ? p->A * profile(p->A_prof, s) : p->A; }

/* ------------------------------------------------------------------------ */
/* WENO5 (Jiang-Shu) reconstruction of one interface from five values        */
/* v[0..4] = v_{-2}, v_{-1}, v_0, v_1, v_2 (upwind side on the left).         */
/* Exposes the three candidate values q, the smoothness indicators beta and   */
/* the reconstructed value, so tests can check each against its definition.   */
/* ------------------------------------------------------------------------ */
void orc_weno_parts(const double *v, double eps, double *q, double *beta, double *fhat)
{
    double vm2 = v[0], vm1 = v[1], v0 = v[2], v1 = v[3], v2 = v[4];
    q[0] = (2.0 * vm2 - 7.0 * vm1 + 11.0 * v0) / 6.0;
    q[1] = (-vm1 + 5.0 * v0 + 2.0 * v1) / 6.0;
    q[2] = (2.0 * v0 + 5.0 * v1 - v2) / 6.0;
    double t;
    t = vm2 - 2.0 * vm1 + v0;   beta[0] = 13.0 / 12.0 * t * t;
    t = vm2 - 4.0 * vm1 + 3.0 * v0; beta[0] += 0.25 * t * t;
    t = vm1 - 2.0 * v0 + v1;    beta[1] = 13.0 / 12.0 * t * t;
    t = vm1 - v1;               beta[1] += 0.25 * t * t;
    t = v0 - 2.0 * v1 + v2;     beta[2] = 13.0 / 12.0 * t * t;
    t = 3.0 * v0 - 4.0 * v1 + v2; beta[2] += 0.25 * t * t;
    const double d[3] = {0.1, 0.6, 0.3};
    double a[3], sa = 0.0;
    for (int r = 0; r < 3; r++) {
        double e = eps + beta[r];
        a[r] = d[r] / (e * e);
        sa += a[r];
    }
    double f = 0.0;
    for (int r = 0; r < 3; r++) f += a[r] / sa * q[r];
    *fhat = f;
}

/* Numerical flux F_hat_{k+1/2} at every interface of one periodic row, for
 * the tau-flux of Eq. 7, f(u) = -c u - (B/2) u^2 with c = 2 pi U_par of the row
 * (c = 0: homogeneous medium). */
static void weno_row_fluxes(const double *u, int n, double c, double B, double alpha, double eps, double *F)
{
    double *fp = (double *)malloc(sizeof(double) * n);
    double *fm = (double *)malloc(sizeof(double) * n);
    for (int i = 0; i < n; i++) {
        double f = -c * u[i] - 0.5 * B * u[i] * u[i];
        fp[i] = 0.5 * (f + alpha * u[i]);        /* Lax-Friedrichs splitting */
        fm[i] = 0.5 * (f - alpha * u[i]);
    }
    for (int k = 0; k < n; k++) {
        double v[5], q[3], be[3], Fp, Fm;
        for (int s = 0; s < 5; s++) v[s] = fp[((k - 2 + s) % n + n) % n];          /* k-2 .. k+2 */
        orc_weno_parts(v, eps, q, be, &Fp);
        for (int s = 0; s < 5; s++) v[s] = fm[((k + 3 - s) % n + n) % n];          /* k+3 .. k-1 */
        orc_weno_parts(v, eps, q, be, &Fm);
        F[k] = Fp + Fm;                          /* interface k + 1/2 */
    }
    free(fp); free(fm);
}

/* Random velocity field of Algorithm 1 at (sigma, y_j) for every row j:
 * U_par, U_perp and d U_perp / d y (the y-derivative of the same sum of
 * modes, differentiated term by term).  All zero without modes. */
void orc_medium(const orc_params *p, double sigma, double *upar, double *uperp, double *duperp)
{
    double dy = (p->y_max - p->y_min) / p->ny;
    for (int j = 0; j < p->ny; j++) {
        double rho = p->y_min + j * dy;
        double r = sqrt(sigma * sigma + rho * rho), psi = atan2(rho, sigma);
        double a = 0.0, b = 0.0, db = 0.0;
        for (int n = 0; n < p->n_modes; n++) {
            double th = p->mode_theta[n];
            /* U~_n = |U~_n| (-sin theta_n, cos theta_n), orthogonal to K_n */
            double u1 = -p->mode_amp[n] * sin(th), u2 = p->mode_amp[n] * cos(th);
            double arg = p->mode_klam[n] * r * cos(th - psi) + p->mode_phase[n];
            a += u1 * cos(arg);
            b += u2 * cos(arg);
            /* d(arg)/d rho = |K_n| lambda sin(theta_n) */
            db += -u2 * sin(arg) * p->mode_klam[n] * sin(th);
        }
        upar[j] = a; uperp[j] = b; duperp[j] = db;
    }
}

/* WENO part of b: b_k = -(F_{k+1/2} - F_{k-1/2}) / dtau, row by row (the
 * tau-flux of Eq. 7), plus, with a random medium, the y-flux U_perp u by
 * WENO5 along y, -(G_{j+1/2} - G_{j-1/2}) / dy, and the source d_y U_perp u
 * (the rewriting of U_perp d_y u that follows Eq. 7). */
void orc_weno_rhs(const orc_params *p, const double *u, double sigma, double *b)
{
    int nx = p->nx, ny = p->ny;
    double dtau = (p->tau_max - p->tau_min) / nx;
    double Bs = orc_B_of(p, sigma);
    double *upar = calloc(ny, sizeof(double)), *uperp = calloc(ny, sizeof(double));
    double *duperp = calloc(ny, sizeof(double));
    if (p->n_modes > 0) orc_medium(p, sigma, upar, uperp, duperp);
    #pragma omp parallel
    {
        double *F = (double *)malloc(sizeof(double) * nx);
        #pragma omp for schedule(static)
        for (int j = 0; j < ny; j++) {
            const double *ur = u + (size_t)j * nx;
            double c = 2.0 * M_PI * upar[j];
            /* global LF speed of the row: |f'(u)| = |c + B u| <= |c| + B M */
            double alpha = fabs(c) + Bs * p->lf_umax;
            weno_row_fluxes(ur, nx, c, Bs, alpha, p->weno_eps, F);
            for (int k = 0; k < nx; k++) b[(size_t)j * nx + k] = -(F[k] - F[(k - 1 + nx) % nx]) / dtau;
        }
        free(F);
    }
    if (p->n_modes > 0) {
        double dy = (p->y_max - p->y_min) / ny;
        double ay = 0.0;                      /* global LF speed along y: max |U_perp| */
        for (int j = 0; j < ny; j++) ay = fmax(ay, fabs(uperp[j]));
        #pragma omp parallel
        {
            double *col = malloc(sizeof(double) * ny), *G = malloc(sizeof(double) * ny);
            #pragma omp for schedule(static)
            for (int k = 0; k < nx; k++) {
                for (int j = 0; j < ny; j++) col[j] = u[(size_t)j * nx + k];
                /* y-flux g(u) = U_perp(y) u, split as (g +- ay u)/2 */
                double *gp = malloc(sizeof(double) * ny), *gm = malloc(sizeof(double) * ny);
                for (int j = 0; j < ny; j++) {
                    double g = uperp[j] * col[j];
                    gp[j] = 0.5 * (g + ay * col[j]);
                    gm[j] = 0.5 * (g - ay * col[j]);
                }
                for (int j = 0; j < ny; j++) {
                    double v[5], q[3], be[3], Gp, Gm;
                    for (int s = 0; s < 5; s++) v[s] = gp[((j - 2 + s) % ny + ny) % ny];
                    orc_weno_parts(v, p->weno_eps, q, be, &Gp);
                    for (int s = 0; s < 5; s++) v[s] = gm[((j + 3 - s) % ny + ny) % ny];
                    orc_weno_parts(v, p->weno_eps, q, be, &Gm);
                    G[j] = Gp + Gm;                   /* interface j + 1/2 */
                }
                for (int j = 0; j < ny; j++)
                    b[(size_t)j * nx + k] += -(G[j] - G[(j - 1 + ny) % ny]) / dy + duperp[j] * col[j];
                free(gp); free(gm);
            }
            free(col); free(G);
        }
    }
    free(upar); free(uperp); free(duperp);
}

/* 2-D spectrum of b(sigma, u) given u and its spectrum:                          */
/* F(b) = F(WENO(u)) - (A(sigma) - A) k_tau^2 F(u).                               */
static void rhs_hat(const orc_params *p, const double *u, const double *ur_hat, const double *ui_hat,
                    double sigma, double *br, double *bi)
{
    size_t N = (size_t)p->nx * p->ny;
    orc_weno_rhs(p, u, sigma, br);
    memset(bi, 0, sizeof(double) * N);
    orc_fft2d(br, bi, p->nx, p->ny, 0);
    double dA = orc_A_of(p, sigma) - p->A;
    if (dA != 0.0) {
        double Lx = p->tau_max - p->tau_min;
        for (int j = 0; j < p->ny; j++)
            for (int m = 0; m < p->nx; m++) {
                double kt = 2.0 * M_PI * signed_index(m, p->nx) / Lx;
                size_t i = (size_t)j * p->nx + m;
                br[i] -= dA * kt * kt * ur_hat[i];
                bi[i] -= dA * kt * kt * ui_hat[i];
            }
    }
}

/* Physical-space b(sigma, u) including the absorption-deviation term. */
void orc_rhs(const orc_params *p, const double *u, double sigma, double *b)
{
    size_t N = (size_t)p->nx * p->ny;
    double *ur = malloc(sizeof(double) * N), *ui = calloc(N, sizeof(double));
    double *bi = malloc(sizeof(double) * N);
    memcpy(ur, u, sizeof(double) * N);
    orc_fft2d(ur, ui, p->nx, p->ny, 0);
    rhs_hat(p, u, ur, ui, sigma, b, bi);
    orc_fft2d(b, bi, p->nx, p->ny, 1);
    free(ur); free(ui); free(bi);
}

/* Diagnostics: mean, energy = dtau dy sum u^2, max |u|, count of non-finite values. */
void orc_diag(const orc_params *p, const double *u, double *out4)
{
    size_t N = (size_t)p->nx * p->ny;
    double s = 0.0, e = 0.0, mx = 0.0, nf = 0.0;
    for (size_t i = 0; i < N; i++) {
        double v = u[i];
        if (!isfinite(v)) { nf += 1.0; continue; }
        s += v; e += v * v;
        if (fabs(v) > mx) mx = fabs(v);
    }
    double dtau = (p->tau_max - p->tau_min) / p->nx, dy = (p->y_max - p->y_min) / p->ny;
    out4[0] = s / (double)N; out4[1] = dtau * dy * e; out4[2] = mx; out4[3] = nf;
}

/* ------------------------------------------------------------------------ */
/* ExpRK22 in Fourier space (Eq. 11 / Algorithm 2).  State kept in physical   */
/* space between steps; the transforms are applied exactly as listed there.   */
/* u: [ny][nx], advanced in place.  u_star (nullable): V^{n,*} of the last    */
/* step.  hist (nullable): [n_steps][4] diagnostics after each step.          */
/* ------------------------------------------------------------------------ */
typedef struct {
    double *Er, *Ei, *P1r, *P1i, *P2r, *P2i;
} tables_t;

static void tables_alloc(const orc_params *p, tables_t *t)
{
    size_t N = (size_t)p->nx * p->ny;
    t->Er = malloc(sizeof(double) * N); t->Ei = malloc(sizeof(double) * N);
    t->P1r = malloc(sizeof(double) * N); t->P1i = malloc(sizeof(double) * N);
    t->P2r = malloc(sizeof(double) * N); t->P2i = malloc(sizeof(double) * N);
    orc_tables(p, t->Er, t->Ei, t->P1r, t->P1i, t->P2r, t->P2i);
}
static void tables_free(tables_t *t)
{
    free(t->Er); free(t->Ei); free(t->P1r); free(t->P1i); free(t->P2r); free(t->P2i);
}

/* One ExpRK22 step. Work arrays are allocated by the caller (7 N doubles). */
static void exprk22_step(const orc_params *p, const tables_t *t, double *u, double sigma,
                         double *u_star_out, double *w)
{
    size_t N = (size_t)p->nx * p->ny;
    double dt = p->dt;
    double *ur = w, *ui = w + N, *b1r = w + 2 * N, *b1i = w + 3 * N;
    double *sr = w + 4 * N, *si = w + 5 * N, *b2i = w + 6 * N;
    /* STEP 1: b(sigma^n, V^n) and its spectrum; F(V^n) */
    memcpy(ur, u, sizeof(double) * N);
    memset(ui, 0, sizeof(double) * N);
    orc_fft2d(ur, ui, p->nx, p->ny, 0);
    rhs_hat(p, u, ur, ui, sigma, b1r, b1i);
    /* STEP 2: F(V*) = E F(V^n) + dt Phi1 F(b1) */
    for (size_t i = 0; i < N; i++) {
        cpx E = c_mk(t->Er[i], t->Ei[i]), P1 = c_mk(t->P1r[i], t->P1i[i]);
        cpx v = c_add(c_mul(E, c_mk(ur[i], ui[i])), c_mul(c_mk(dt * P1.re, dt * P1.im), c_mk(b1r[i], b1i[i])));
        sr[i] = v.re; si[i] = v.im;
    }
    orc_fft2d(sr, si, p->nx, p->ny, 1);          /* V* = Re F^{-1}(...) */
    double *vs = malloc(sizeof(double) * N);
    memcpy(vs, sr, sizeof(double) * N);
    if (u_star_out) memcpy(u_star_out, vs, sizeof(double) * N);
    /* STEP 3: b(sigma^{n+1}, V*) and its spectrum */
    memset(si, 0, sizeof(double) * N);
    orc_fft2d(sr, si, p->nx, p->ny, 0);          /* F(V*) */
    double *b2r = malloc(sizeof(double) * N);
    rhs_hat(p, vs, sr, si, sigma + dt, b2r, b2i);
    /* STEP 4: F(V^{n+1}) = E F(V^n) + dt [ (Phi1 - Phi2) F(b1) + Phi2 F(b2) ] */
    for (size_t i = 0; i < N; i++) {
        cpx E = c_mk(t->Er[i], t->Ei[i]);
        cpx P1 = c_mk(t->P1r[i], t->P1i[i]), P2 = c_mk(t->P2r[i], t->P2i[i]);
        cpx acc = c_mul(E, c_mk(ur[i], ui[i]));
        cpx d = c_sub(P1, P2);
        cpx tb = c_add(c_mul(d, c_mk(b1r[i], b1i[i])), c_mul(P2, c_mk(b2r[i], b2i[i])));
        acc = c_add(acc, c_mk(dt * tb.re, dt * tb.im));
        sr[i] = acc.re; si[i] = acc.im;
    }
    orc_fft2d(sr, si, p->nx, p->ny, 1);
    for (size_t i = 0; i < N; i++) u[i] = sr[i];
    free(vs); free(b2r);
}

/* One exponential Euler step (Sec. 3.2): F(V^{n+1}) = E F(V^n) + dt Phi1 F(b(sigma^n, V^n)),
 * i.e. the first stage of Eq. 5 taken as the step. */
static void expeuler_step(const orc_params *p, const tables_t *t, double *u, double sigma, double *w)
{
    size_t N = (size_t)p->nx * p->ny;
    double dt = p->dt;
    double *ur = w, *ui = w + N, *b1r = w + 2 * N, *b1i = w + 3 * N, *sr = w + 4 * N, *si = w + 5 * N;
    memcpy(ur, u, sizeof(double) * N);
    memset(ui, 0, sizeof(double) * N);
    orc_fft2d(ur, ui, p->nx, p->ny, 0);
    rhs_hat(p, u, ur, ui, sigma, b1r, b1i);
    for (size_t i = 0; i < N; i++) {
        cpx E = c_mk(t->Er[i], t->Ei[i]), P1 = c_mk(t->P1r[i], t->P1i[i]);
        cpx v = c_add(c_mul(E, c_mk(ur[i], ui[i])), c_mul(c_mk(dt * P1.re, dt * P1.im), c_mk(b1r[i], b1i[i])));
        sr[i] = v.re; si[i] = v.im;
    }
    orc_fft2d(sr, si, p->nx, p->ny, 1);
    memcpy(u, sr, sizeof(double) * N);
}

/* One step of the plan's method; u_star_out (nullable): V^{n,*} (the Euler
 * step itself for method 1). */
static void one_step(const orc_params *p, const tables_t *t, double *u, double sigma, double *u_star_out, double *w)
{
    if (p->method == 1) {
        expeuler_step(p, t, u, sigma, w);
        if (u_star_out) memcpy(u_star_out, u, sizeof(double) * (size_t)p->nx * p->ny);
    } else {
        exprk22_step(p, t, u, sigma, u_star_out, w);
    }
}

int orc_run(const orc_params *p, double *u, int64_t n_steps, double sigma0, double *u_star, double *hist)
{
    size_t N = (size_t)p->nx * p->ny;
    tables_t t;
    tables_alloc(p, &t);
    double *w = malloc(sizeof(double) * 7 * N);
    for (int64_t n = 0; n < n_steps; n++) {
        double sigma = sigma0 + (double)n * p->dt;
        one_step(p, &t, u, sigma, u_star, w);
        if (hist) orc_diag(p, u, hist + 4 * n);
    }
    free(w);
    tables_free(&t);
    return 0;
}

/* Same as orc_run, also returning the wall time of every step in
   step_seconds[n] (table set-up excluded): used to time the oracle as a CPU
   baseline; the arithmetic is that of orc_run. */
#include <time.h>
int orc_run_timed(const orc_params *p, double *u, int64_t n_steps, double sigma0, double *step_seconds)
{
    size_t N = (size_t)p->nx * p->ny;
    tables_t t;
    tables_alloc(p, &t);
    double *w = malloc(sizeof(double) * 7 * N);
    for (int64_t n = 0; n < n_steps; n++) {
        struct timespec a, b;
        clock_gettime(CLOCK_MONOTONIC, &a);
        one_step(p, &t, u, sigma0 + (double)n * p->dt, NULL, w);
        clock_gettime(CLOCK_MONOTONIC, &b);
        step_seconds[n] = (double)(b.tv_sec - a.tv_sec) + 1e-9 * (double)(b.tv_nsec - a.tv_nsec);
    }
    free(w);
    tables_free(&t);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Adjoint.  With P_X := Re F^{-1} diag(X) F (a real operator for the         */
/* Hermitian-symmetric tables of Eq. 11), one step reads                      */
/*    b1 = G_n(u),  u* = P_E u + P_{dt Phi1} b1,  b2 = G_{n+1}(u*),             */
/*    u' = u* + P_{dt Phi2} (b2 - b1),                                          */
/* with G_s(u) = WENO_s(u) + (A(s) - A) d_tau^2 u.  Its transpose, for a       */
/* cotangent lam' of u', is                                                    */
/*    mu2 = P_{conj(dt Phi2)} lam',  lam* = lam' + J_{G_{n+1}}(u*)^T mu2,      */
/*    nu1 = P_{conj(dt Phi1)} lam* - mu2,                                       */
/*    lam = P_{conj E} lam* + J_{G_n}(u)^T nu1.                                 */
/* The WENO Jacobian is differentiated analytically through the nonlinear      */
/* weights: with omega_r = a_r / sum a, a_r = d_r/(eps+beta_r)^2,              */
/*    dF/dv_j = sum_r omega_r dq_r/dv_j                                         */
/*              - 2 sum_r omega_r (q_r - F)/(eps+beta_r) dbeta_r/dv_j.          */
/* ------------------------------------------------------------------------ */

/* Gradient of the one-interface reconstruction w.r.t. v[0..4]. */
void orc_weno_grad(const double *v, double eps, double *g)
{
    double q[3], beta[3], F;
    orc_weno_parts(v, eps, q, beta, &F);
    const double d[3] = {0.1, 0.6, 0.3};
    double a[3], sa = 0.0;
    for (int r = 0; r < 3; r++) { double e = eps + beta[r]; a[r] = d[r] / (e * e); sa += a[r]; }
    double om[3];
    for (int r = 0; r < 3; r++) om[r] = a[r] / sa;
    /* dq_r/dv_j */
    const double dq[3][5] = {
        {2.0 / 6.0, -7.0 / 6.0, 11.0 / 6.0, 0.0, 0.0},
        {0.0, -1.0 / 6.0, 5.0 / 6.0, 2.0 / 6.0, 0.0},
        {0.0, 0.0, 2.0 / 6.0, 5.0 / 6.0, -1.0 / 6.0}};
    /* dbeta_r/dv_j from the quadratic forms of the smoothness indicators */
    double db[3][5];
    memset(db, 0, sizeof(db));
    {
        double s = v[0] - 2 * v[1] + v[2], t = v[0] - 4 * v[1] + 3 * v[2];
        double cs = 2.0 * 13.0 / 12.0 * s, ct = 2.0 * 0.25 * t;
        db[0][0] = cs * 1 + ct * 1; db[0][1] = cs * -2 + ct * -4; db[0][2] = cs * 1 + ct * 3;
    }
    {
        double s = v[1] - 2 * v[2] + v[3], t = v[1] - v[3];
        double cs = 2.0 * 13.0 / 12.0 * s, ct = 2.0 * 0.25 * t;
        db[1][1] = cs * 1 + ct * 1; db[1][2] = cs * -2; db[1][3] = cs * 1 + ct * -1;
    }
    {
        double s = v[2] - 2 * v[3] + v[4], t = 3 * v[2] - 4 * v[3] + v[4];
        double cs = 2.0 * 13.0 / 12.0 * s, ct = 2.0 * 0.25 * t;
        db[2][2] = cs * 1 + ct * 3; db[2][3] = cs * -2 + ct * -4; db[2][4] = cs * 1 + ct * 1;
    }
    for (int j = 0; j < 5; j++) {
        double acc = 0.0;
        for (int r = 0; r < 3; r++) acc += om[r] * dq[r][j];
        for (int r = 0; r < 3; r++) acc += -2.0 * om[r] * (q[r] - F) / (eps + beta[r]) * db[r][j];
        g[j] = acc;
    }
}

/* J_WENO(u)^T mu, physical space, row by row. */
void orc_weno_rhs_T(const orc_params *p, const double *u, double sigma, const double *mu, double *out)
{
    int nx = p->nx, ny = p->ny;
    double dtau = (p->tau_max - p->tau_min) / nx;
    double Bs = orc_B_of(p, sigma);
    double *upar = calloc(ny, sizeof(double)), *uperp = calloc(ny, sizeof(double));
    double *duperp = calloc(ny, sizeof(double));
    if (p->n_modes > 0) orc_medium(p, sigma, upar, uperp, duperp);
    #pragma omp parallel
    {
        double *fp = malloc(sizeof(double) * nx), *fm = malloc(sizeof(double) * nx);
        double *dfp = malloc(sizeof(double) * nx), *dfm = malloc(sizeof(double) * nx);
        #pragma omp for schedule(static)
        for (int j = 0; j < ny; j++) {
            const double *ur = u + (size_t)j * nx;
            const double *mr = mu + (size_t)j * nx;
            double *o = out + (size_t)j * nx;
            /* tau-flux f = -c u - B u^2 / 2 (c = 2 pi U_par of the row), LF speed |c| + B M */
            double c = 2.0 * M_PI * upar[j];
            double alpha = fabs(c) + Bs * p->lf_umax;
            for (int i = 0; i < nx; i++) {
                double f = -c * ur[i] - 0.5 * Bs * ur[i] * ur[i];
                fp[i] = 0.5 * (f + alpha * ur[i]);  fm[i] = 0.5 * (f - alpha * ur[i]);
                dfp[i] = 0.5 * (-c - Bs * ur[i] + alpha); dfm[i] = 0.5 * (-c - Bs * ur[i] - alpha);
                o[i] = 0.0;
            }
            for (int k = 0; k < nx; k++) {
                /* b_k = -(F_{k+1/2} - F_{k-1/2})/dtau, so F_{k+1/2} enters b_k with -1/dtau
                   and b_{k+1} with +1/dtau */
                double psi = (mr[(k + 1) % nx] - mr[k]) / dtau;
                double v[5], g[5];
                for (int s = 0; s < 5; s++) v[s] = fp[((k - 2 + s) % nx + nx) % nx];
                orc_weno_grad(v, p->weno_eps, g);
                for (int s = 0; s < 5; s++) { int i = ((k - 2 + s) % nx + nx) % nx; o[i] += psi * g[s] * dfp[i]; }
                for (int s = 0; s < 5; s++) v[s] = fm[((k + 3 - s) % nx + nx) % nx];
                orc_weno_grad(v, p->weno_eps, g);
                for (int s = 0; s < 5; s++) { int i = ((k + 3 - s) % nx + nx) % nx; o[i] += psi * g[s] * dfm[i]; }
            }
        }
        free(fp); free(fm); free(dfp); free(dfm);
    }
    if (p->n_modes > 0) {
        /* y-flux g = U_perp u split by ay = max |U_perp| (dg+-/du = (U_perp +- ay)/2,
         * constant in u), transposed column by column, plus the source d_y U_perp */
        double dy = (p->y_max - p->y_min) / ny;
        double ay = 0.0;
        for (int j = 0; j < ny; j++) ay = fmax(ay, fabs(uperp[j]));
        #pragma omp parallel
        {
            double *gp = malloc(sizeof(double) * ny), *gm = malloc(sizeof(double) * ny);
            #pragma omp for schedule(static)
            for (int k = 0; k < nx; k++) {
                for (int j = 0; j < ny; j++) {
                    double uu = u[(size_t)j * nx + k], g = uperp[j] * uu;
                    gp[j] = 0.5 * (g + ay * uu);
                    gm[j] = 0.5 * (g - ay * uu);
                }
                for (int j = 0; j < ny; j++) {
                    double psi = (mu[(size_t)((j + 1) % ny) * nx + k] - mu[(size_t)j * nx + k]) / dy;
                    double v[5], g[5];
                    for (int s = 0; s < 5; s++) v[s] = gp[((j - 2 + s) % ny + ny) % ny];
                    orc_weno_grad(v, p->weno_eps, g);
                    for (int s = 0; s < 5; s++) {
                        int i = ((j - 2 + s) % ny + ny) % ny;
                        out[(size_t)i * nx + k] += psi * g[s] * 0.5 * (uperp[i] + ay);
                    }
                    for (int s = 0; s < 5; s++) v[s] = gm[((j + 3 - s) % ny + ny) % ny];
                    orc_weno_grad(v, p->weno_eps, g);
                    for (int s = 0; s < 5; s++) {
                        int i = ((j + 3 - s) % ny + ny) % ny;
                        out[(size_t)i * nx + k] += psi * g[s] * 0.5 * (uperp[i] - ay);
                    }
                }
            }
            free(gp); free(gm);
        }
        for (int j = 0; j < ny; j++)
            for (int k = 0; k < nx; k++) out[(size_t)j * nx + k] += duperp[j] * mu[(size_t)j * nx + k];
    }
    free(upar); free(uperp); free(duperp);
}

/* out = Re F^{-1}( M o F(x) ), M given as re/im arrays, conj selects conj(M). */
static void apply_mult(const orc_params *p, const double *x, const double *Mr, const double *Mi,
                       double scale, int conj, double *out)
{
    size_t N = (size_t)p->nx * p->ny;
    double *re = malloc(sizeof(double) * N), *im = calloc(N, sizeof(double));
    memcpy(re, x, sizeof(double) * N);
    orc_fft2d(re, im, p->nx, p->ny, 0);
    for (size_t i = 0; i < N; i++) {
        cpx m = c_mk(scale * Mr[i], scale * (conj ? -Mi[i] : Mi[i]));
        cpx v = c_mul(m, c_mk(re[i], im[i]));
        re[i] = v.re; im[i] = v.im;
    }
    orc_fft2d(re, im, p->nx, p->ny, 1);
    memcpy(out, re, sizeof(double) * N);
    free(re); free(im);
}

/* J_G(u)^T mu = J_WENO(u)^T mu + (A(s) - A) D2 mu (D2 symmetric). */
static void rhs_T(const orc_params *p, const double *u, double sigma, const double *mu, double *out)
{
    size_t N = (size_t)p->nx * p->ny;
    orc_weno_rhs_T(p, u, sigma, mu, out);
    double dA = orc_A_of(p, sigma) - p->A;
    if (dA != 0.0) {
        double *re = malloc(sizeof(double) * N), *im = calloc(N, sizeof(double));
        memcpy(re, mu, sizeof(double) * N);
        orc_fft2d(re, im, p->nx, p->ny, 0);
        double Lx = p->tau_max - p->tau_min;
        for (int j = 0; j < p->ny; j++)
            for (int m = 0; m < p->nx; m++) {
                double kt = 2.0 * M_PI * signed_index(m, p->nx) / Lx;
                size_t i = (size_t)j * p->nx + m;
                re[i] *= -dA * kt * kt; im[i] *= -dA * kt * kt;
            }
        orc_fft2d(re, im, p->nx, p->ny, 1);
        for (size_t i = 0; i < N; i++) out[i] += re[i];
        free(re); free(im);
    }
}

/* Gradient of a loss w.r.t. u0 given its gradient g_end w.r.t. u(sigma0 + n dt).
   All stage states are stored (no checkpointing): plain reverse sweep. */
int orc_adjoint(const orc_params *p, const double *u0, const double *g_end, int64_t n_steps,
                double sigma0, double *g0)
{
    size_t N = (size_t)p->nx * p->ny;
    tables_t t;
    tables_alloc(p, &t);
    double *w = malloc(sizeof(double) * 7 * N);
    double *us = malloc(sizeof(double) * N * (size_t)(n_steps + 1));
    double *uss = malloc(sizeof(double) * N * (size_t)(n_steps > 0 ? n_steps : 1));
    memcpy(us, u0, sizeof(double) * N);
    for (int64_t n = 0; n < n_steps; n++) {
        memcpy(us + (size_t)(n + 1) * N, us + (size_t)n * N, sizeof(double) * N);
        one_step(p, &t, us + (size_t)(n + 1) * N, sigma0 + n * p->dt, uss + (size_t)n * N, w);
    }
    double *lam = malloc(sizeof(double) * N), *mu2 = malloc(sizeof(double) * N);
    double *lst = malloc(sizeof(double) * N), *tmp = malloc(sizeof(double) * N);
    double *nu1 = malloc(sizeof(double) * N);
    memcpy(lam, g_end, sizeof(double) * N);
    for (int64_t n = n_steps - 1; n >= 0; n--) {
        double sigma = sigma0 + n * p->dt;
        const double *un = us + (size_t)n * N, *ust = uss + (size_t)n * N;
        if (p->method == 1) {
            /* transpose of u' = P_E u + P_{dt Phi1} G_n(u) */
            apply_mult(p, lam, t.P1r, t.P1i, p->dt, 1, nu1);
            apply_mult(p, lam, t.Er, t.Ei, 1.0, 1, lst);
            rhs_T(p, un, sigma, nu1, tmp);
            for (size_t i = 0; i < N; i++) lam[i] = lst[i] + tmp[i];
            continue;
        }
        apply_mult(p, lam, t.P2r, t.P2i, p->dt, 1, mu2);             /* mu2 */
        rhs_T(p, ust, sigma + p->dt, mu2, tmp);                        /* J_{G_{n+1}}(u*)^T mu2 */
        for (size_t i = 0; i < N; i++) lst[i] = lam[i] + tmp[i];       /* lam* */
        apply_mult(p, lst, t.P1r, t.P1i, p->dt, 1, nu1);
        for (size_t i = 0; i < N; i++) nu1[i] -= mu2[i];               /* nu1 */
        apply_mult(p, lst, t.Er, t.Ei, 1.0, 1, lam);                   /* P_{conj E} lam* */
        rhs_T(p, un, sigma, nu1, tmp);
        for (size_t i = 0; i < N; i++) lam[i] += tmp[i];
    }
    memcpy(g0, lam, sizeof(double) * N);
    free(lam); free(mu2); free(lst); free(tmp); free(nu1);
    free(us); free(uss); free(w);
    tables_free(&t);
    return 0;
}
