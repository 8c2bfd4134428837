/*
 * oracle.c -- plain, slow FP64 CPU oracle for the 1D swept stencil path.
 *
 * TEST INFRASTRUCTURE. Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg load this library. The CUDA path never calls it,
 * shares no code with it, and must fail loudly when its own extension is absent.
 *
 * What is computed here is the plain definition of each scheme: a naive
 * time-step loop over the whole grid, evaluated from the old time level for
 * every cell, with no tiles, no swept phases and no reordering. The swept rule
 * (Section 4.1 of Magee, Walker & Niemeyer, "Applying the swept rule for solving
 * explicit partial differential equations on heterogeneous computing systems")
 * states that swept and classic decompositions use the same numerical method, so
 * this naive loop is the reference result for both.
 *
 * The paper names its schemes but does not print them (Section 4.2: FTCS heat
 * equation; second-order finite-volume Euler scheme with a minmod limiter). The
 * readings written out below are the project's fixed definition of those
 * schemes; each function states which reading it follows.
 *
 * Rounding: textbook expressions, compiled with -ffp-contract=off so that no
 * multiply-add is fused. Loops over cells may run in parallel (OpenMP); every
 * cell is computed independently from the old level, so the result does not
 * depend on the thread count.
 *
 * Parity status per function (see the pins in tests/test_oracle_*.py):
 *   orc_heat_run          pinned (closed form, matrix power, conservation)
 *   orc_heat_modes        pinned (matrix power, initial state, zero mode)
 *   orc_euler_run         pinned (constant state, conservation, mirror symmetry,
 *                          Sod convergence, smooth-wave convergence order)
 *   orc_riemann_star /
 *   orc_riemann_sample    pinned (Rankine-Hugoniot and isentropic relations,
 *                          symmetric and trivial cases)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PERIODIC 0
#define ORC_TRANSMISSIVE 1

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the parallel cell loops from here on (timing of the 1-core rate;
 * small grids). Results do not depend on it: every cell is computed alone. */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Heat equation, FTCS (Section 4.2: first-order forward in time, central in
 * space). Reading: u_j <- u_j + r*((u_{j-1} + u_{j+1}) - 2 u_j), r = alpha dt/dx^2,
 * all cells from the old level. Periodic: indices wrap. Transmissive
 * (zero-gradient): the ghost beyond each end copies the end cell.            */
/* ------------------------------------------------------------------------ */
int orc_heat_run(int64_t n, double r, int boundary, int64_t nsteps, double *u)
{
    if (n < 2 || nsteps < 0 || !u) return -1;
    double *v = (double *)malloc((size_t)n * sizeof(double));
    if (!v) return -2;
    double *cur = u, *nxt = v;
    for (int64_t s = 0; s < nsteps; ++s) {
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < n; ++j) {
            double left, right;
            if (j > 0) left = cur[j - 1];
            else left = (boundary == ORC_PERIODIC) ? cur[n - 1] : cur[0];
            if (j < n - 1) right = cur[j + 1];
            else right = (boundary == ORC_PERIODIC) ? cur[0] : cur[n - 1];
            nxt[j] = cur[j] + r * ((left + right) - 2.0 * cur[j]);
        }
        double *t = cur; cur = nxt; nxt = t;
    }
    if (cur != u) memcpy(u, cur, (size_t)n * sizeof(double));
    free(v);
    return 0;
}

/* Exact discrete solution of FTCS on a periodic grid for an initial state that
 * is a sum of sine modes u_j = sum_m a_m sin(2 pi k_m j / n): each mode is an
 * eigenvector of the FTCS operator with eigenvalue G(k) = 1 - 4 r sin^2(pi k/n),
 * so u_j^s = sum_m a_m G(k_m)^s sin(2 pi k_m j / n). Evaluated in long double.
 * Output at the cell indices idx[0..nidx).                                   */
int orc_heat_modes(int64_t n, double r, int64_t nsteps, int nmodes,
                   const double *amp, const int64_t *k,
                   const int64_t *idx, int64_t nidx, double *out)
{
    if (n < 1 || nmodes < 0 || nidx < 0) return -1;
    const long double pi = acosl(-1.0L);
    for (int64_t q = 0; q < nidx; ++q) {
        long double sum = 0.0L;
        for (int m = 0; m < nmodes; ++m) {
            long double sk = sinl(pi * (long double)k[m] / (long double)n);
            long double dec = 4.0L * (long double)r * sk * sk;  /* 1 - G */
            long double g = 1.0L - dec;
            long double gs;
            if (nsteps == 0) gs = 1.0L;
            else if (g > 0.0L) gs = expl((long double)nsteps * log1pl(-dec));
            else gs = powl(g, (long double)nsteps);
            /* angle reduced exactly in integers before scaling */
            int64_t kj = (int64_t)(((__int128)k[m] * idx[q]) % n);
            if (kj < 0) kj += n;
            long double ang = 2.0L * pi * (long double)kj / (long double)n;
            sum += (long double)amp[m] * gs * sinl(ang);
        }
        out[q] = (double)sum;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Heat equation in two dimensions, FTCS with the 5-point stencil: the 2D
 * extension of the swept rule that Section 6 names as future work. Reading:
 *   u_ij <- u_ij + ( rx*((u_{i-1,j} + u_{i+1,j}) - 2 u_ij)
 *                  + ry*((u_{i,j-1} + u_{i,j+1}) - 2 u_ij) ),
 * every cell from the old level; u[j*nx + i], i along x (fastest). Periodic:
 * indices wrap in both directions; transmissive: a ghost copies the edge cell.
 * Written so that swapping x and y (and rx, ry) transposes the result bit for bit,
 * and a state constant along y evolves, row by row, bit for bit as orc_heat_run
 * with r = rx (the y-difference is then exactly zero).                       */
/* ------------------------------------------------------------------------ */
int orc_heat2d_run(int64_t nx, int64_t ny, double rx, double ry, int boundary, int64_t nsteps, double *u)
{
    if (nx < 2 || ny < 2 || nsteps < 0 || !u) return -1;
    const int64_t n = nx * ny;
    double *v = (double *)malloc((size_t)n * sizeof(double));
    if (!v) return -2;
    double *cur = u, *nxt = v;
    const int per = boundary == ORC_PERIODIC;
    for (int64_t s = 0; s < nsteps; ++s) {
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < ny; ++j) {
            const int64_t jd = j > 0 ? j - 1 : (per ? ny - 1 : 0);
            const int64_t ju = j < ny - 1 ? j + 1 : (per ? 0 : ny - 1);
            for (int64_t i = 0; i < nx; ++i) {
                const int64_t il = i > 0 ? i - 1 : (per ? nx - 1 : 0);
                const int64_t ir = i < nx - 1 ? i + 1 : (per ? 0 : nx - 1);
                const double c = cur[j * nx + i];
                const double xd = (cur[j * nx + il] + cur[j * nx + ir]) - 2.0 * c;
                const double yd = (cur[jd * nx + i] + cur[ju * nx + i]) - 2.0 * c;
                nxt[j * nx + i] = c + (rx * xd + ry * yd);
            }
        }
        double *t = cur; cur = nxt; nxt = t;
    }
    if (cur != u) memcpy(u, cur, (size_t)n * sizeof(double));
    free(v);
    return 0;
}

/* Exact discrete solution of 2D FTCS on a periodic nx x ny grid for a sum of
 * separable modes u_ij = sum_m a_m f_m(2 pi kx_m i / nx) g_m(2 pi ky_m j / ny),
 * f, g = sin (flag 0) or cos (flag 1). Each such product is an eigenvector of the
 * 5-point operator: the x-difference of sin/cos(theta i) is (2 cos theta - 2)
 * times it, so G = 1 - 4 rx sin^2(pi kx/nx) - 4 ry sin^2(pi ky/ny) and
 * u^s = sum_m a_m G_m^s f_m g_m. Long double; output at cells (ii[q], jj[q]).  */
int orc_heat2d_modes(int64_t nx, int64_t ny, double rx, double ry, int64_t nsteps, int nmodes,
                     const double *amp, const int64_t *kx, const int64_t *ky, const int32_t *fx,
                     const int32_t *fy, const int64_t *ii, const int64_t *jj, int64_t nidx, double *out)
{
    if (nx < 1 || ny < 1 || nmodes < 0 || nidx < 0) return -1;
    const long double pi = acosl(-1.0L);
    for (int64_t q = 0; q < nidx; ++q) {
        long double sum = 0.0L;
        for (int m = 0; m < nmodes; ++m) {
            const long double sx = sinl(pi * (long double)kx[m] / (long double)nx);
            const long double sy = sinl(pi * (long double)ky[m] / (long double)ny);
            const long double g = 1.0L - 4.0L * (long double)rx * sx * sx - 4.0L * (long double)ry * sy * sy;
            const long double gs = nsteps == 0 ? 1.0L : powl(g, (long double)nsteps);
            int64_t ki = (int64_t)(((__int128)kx[m] * ii[q]) % nx);
            int64_t kj = (int64_t)(((__int128)ky[m] * jj[q]) % ny);
            if (ki < 0) ki += nx;
            if (kj < 0) kj += ny;
            const long double ax = 2.0L * pi * (long double)ki / (long double)nx;
            const long double ay = 2.0L * pi * (long double)kj / (long double)ny;
            const long double f = fx[m] ? cosl(ax) : sinl(ax);
            const long double h = fy[m] ? cosl(ay) : sinl(ay);
            sum += (long double)amp[m] * gs * f * h;
        }
        out[q] = (double)sum;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Euler equations, second-order finite volume with a minmod limiter driven by
 * the pressure ratio (Section 4.2; Section 4.3 / Fig. 2: the state carries
 * Q = {rho, rho u, E} and a pressure ratio, a predictor stage assigns and a
 * final stage adds). Reading used here (fixed project definition):
 *   p = (gamma-1) (E - 1/2 m u),  u = m / rho
 *   theta_i = (p_i - p_{i-1}) / (p_{i+1} - p_i) when both differences are
 *             nonzero with equal sign, else 0
 *   phi(theta) = min(1, theta); phit(theta) = 1 if 0 < theta <= 1,
 *                1/theta if theta > 1, 0 if theta == 0
 *   face i+1/2:  QL = Q_i + 1/2 phi(theta_i) (Q_{i+1} - Q_i)
 *                QR = Q_{i+1} - 1/2 phit(theta_{i+1}) (Q_{i+1} - Q_i)
 *   flux (Rusanov / local Lax-Friedrichs):
 *     Fh = 1/2 (F(QL) + F(QR)) - 1/2 s (QR - QL),  s = max(|uL|+cL, |uR|+cR)
 *     F(Q) = (m, m u + p, (E + p) u),  c = sqrt(gamma p / rho)
 *   predictor: Q* = Q^n - (lambda/2) (Fh_{i+1/2}(Q^n) - Fh_{i-1/2}(Q^n))
 *   final:     Q^{n+1} = Q^n - lambda (Fh_{i+1/2}(Q*) - Fh_{i-1/2}(Q*))
 *   lambda = dt/dx. Transmissive ends: ghost states copy the end cells (their
 *   pressure ratio is 0); periodic ends wrap.                               */
/* ------------------------------------------------------------------------ */
static double orc_pressure(double gamma, double rho, double m, double E)
{
    double u = m / rho;
    return (gamma - 1.0) * (E - 0.5 * m * u);
}

static double orc_ratio(double pm, double p0, double pp)
{
    double dm = p0 - pm;
    double dp = pp - p0;
    if ((dm > 0.0 && dp > 0.0) || (dm < 0.0 && dp < 0.0)) return dm / dp;
    return 0.0;
}

static double orc_phi(double th) { return th < 1.0 ? th : 1.0; }

static double orc_phit(double th)
{
    if (th > 1.0) return 1.0 / th;
    if (th > 0.0) return 1.0;
    return 0.0;
}

static void orc_phys_flux(double gamma, const double q[3], double f[3], double *speed)
{
    double rho = q[0], m = q[1], E = q[2];
    double u = m / rho;
    double p = (gamma - 1.0) * (E - 0.5 * m * u);
    double c = sqrt(gamma * p / rho);
    f[0] = m;
    f[1] = m * u + p;
    f[2] = (E + p) * u;
    *speed = fabs(u) + c;
}

/* Numerical flux at the face between cell a (left) and cell b (right). */
static void orc_face_flux(double gamma, const double qa[3], double tha,
                          const double qb[3], double thb, double out[3])
{
    double phl = orc_phi(tha), phr = orc_phit(thb);
    double ql[3], qr[3], fl[3], fr[3], sl, sr;
    for (int c = 0; c < 3; ++c) {
        double d = qb[c] - qa[c];
        ql[c] = qa[c] + 0.5 * phl * d;
        qr[c] = qb[c] - 0.5 * phr * d;
    }
    orc_phys_flux(gamma, ql, fl, &sl);
    orc_phys_flux(gamma, qr, fr, &sr);
    double s = sl > sr ? sl : sr;
    for (int c = 0; c < 3; ++c)
        out[c] = 0.5 * (fl[c] + fr[c]) - 0.5 * s * (qr[c] - ql[c]);
}

/* One stage: fluxes of state qin (3 planes of n) at all n+1 faces.
 * Face f lies between cell f-1 and cell f. Work arrays: p, th (n), fh (3(n+1)). */
static void orc_stage_fluxes(int64_t n, double gamma, int boundary,
                             double *const qin[3], double *p, double *th, double *fh)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        p[i] = orc_pressure(gamma, qin[0][i], qin[1][i], qin[2][i]);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double pm, pp;
        if (i > 0) pm = p[i - 1];
        else pm = (boundary == ORC_PERIODIC) ? p[n - 1] : p[0];
        if (i < n - 1) pp = p[i + 1];
        else pp = (boundary == ORC_PERIODIC) ? p[0] : p[n - 1];
        th[i] = orc_ratio(pm, p[i], pp);
    }
#pragma omp parallel for schedule(static)
    for (int64_t f = 0; f <= n; ++f) {
        int64_t a = f - 1, b = f;
        double tha, thb;
        if (a < 0) {
            a = (boundary == ORC_PERIODIC) ? n - 1 : 0;
            tha = (boundary == ORC_PERIODIC) ? th[a] : 0.0;
        } else {
            tha = th[a];
        }
        if (b >= n) {
            b = (boundary == ORC_PERIODIC) ? 0 : n - 1;
            thb = (boundary == ORC_PERIODIC) ? th[b] : 0.0;
        } else {
            thb = th[b];
        }
        double qa[3] = {qin[0][a], qin[1][a], qin[2][a]};
        double qb[3] = {qin[0][b], qin[1][b], qin[2][b]};
        double out[3];
        orc_face_flux(gamma, qa, tha, qb, thb, out);
        fh[3 * f + 0] = out[0];
        fh[3 * f + 1] = out[1];
        fh[3 * f + 2] = out[2];
    }
}

int orc_euler_run(int64_t n, double lambda, double gamma, int boundary,
                  int64_t nsteps, double *rho, double *mom, double *ene)
{
    if (n < 2 || nsteps < 0 || !rho || !mom || !ene) return -1;
    double *p = (double *)malloc((size_t)n * sizeof(double));
    double *th = (double *)malloc((size_t)n * sizeof(double));
    double *fh = (double *)malloc((size_t)(n + 1) * 3 * sizeof(double));
    double *qs = (double *)malloc((size_t)n * 3 * sizeof(double));
    if (!p || !th || !fh || !qs) { free(p); free(th); free(fh); free(qs); return -2; }
    double *q[3] = {rho, mom, ene};
    double *qstar[3] = {qs, qs + n, qs + 2 * n};
    const double half_lambda = 0.5 * lambda;
    for (int64_t s = 0; s < nsteps; ++s) {
        /* predictor */
        orc_stage_fluxes(n, gamma, boundary, q, p, th, fh);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i)
            for (int c = 0; c < 3; ++c)
                qstar[c][i] = q[c][i] - half_lambda * (fh[3 * (i + 1) + c] - fh[3 * i + c]);
        /* final */
        orc_stage_fluxes(n, gamma, boundary, qstar, p, th, fh);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i)
            for (int c = 0; c < 3; ++c)
                q[c][i] = q[c][i] - lambda * (fh[3 * (i + 1) + c] - fh[3 * i + c]);
    }
    free(p); free(th); free(fh); free(qs);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Exact solution of the Riemann problem for the 1D Euler equations of an ideal
 * gas (the textbook construction: a pressure function summing the left and
 * right wave relations, solved by Newton iteration for the star pressure, then
 * sampled on x/t). Used to pin the Euler oracle on the Sod shock tube.       */
/* ------------------------------------------------------------------------ */
typedef struct { double rho, u, p, c; } orc_side;

/* Velocity change across the wave on one side as a function of the star
 * pressure, and its derivative. Shock branch: Rankine-Hugoniot; rarefaction
 * branch: isentropic with the generalised Riemann invariant.                 */
static double orc_wave_fn(double ps, const orc_side *k, double gamma, double *deriv)
{
    if (ps > k->p) {
        double a = 2.0 / ((gamma + 1.0) * k->rho);
        double b = (gamma - 1.0) / (gamma + 1.0) * k->p;
        double q = sqrt(a / (ps + b));
        *deriv = q * (1.0 - 0.5 * (ps - k->p) / (b + ps));
        return (ps - k->p) * q;
    } else {
        double e = (gamma - 1.0) / (2.0 * gamma);
        double pr = ps / k->p;
        *deriv = 1.0 / (k->rho * k->c) * pow(pr, -(gamma + 1.0) / (2.0 * gamma));
        return 2.0 * k->c / (gamma - 1.0) * (pow(pr, e) - 1.0);
    }
}

/* out: p*, u*, rho*_L, rho*_R. Returns 0, or -1 when the data create vacuum. */
int orc_riemann_star(double rl, double ul, double pl, double rr, double ur, double pr,
                     double gamma, double *out)
{
    orc_side L = {rl, ul, pl, sqrt(gamma * pl / rl)};
    orc_side R = {rr, ur, pr, sqrt(gamma * pr / rr)};
    if (2.0 * (L.c + R.c) / (gamma - 1.0) <= ur - ul) return -1;
    /* start from the primitive-variable linearisation, kept positive */
    double ps = 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (L.c + R.c);
    if (ps < 1e-8) ps = 1e-8;
    for (int it = 0; it < 200; ++it) {
        double dl, dr;
        double f = orc_wave_fn(ps, &L, gamma, &dl) + orc_wave_fn(ps, &R, gamma, &dr) + (ur - ul);
        double pn = ps - f / (dl + dr);
        if (pn < 1e-14) pn = 1e-14;
        double change = 2.0 * fabs(pn - ps) / (pn + ps);
        ps = pn;
        if (change < 1e-15) break;
    }
    double dl, dr;
    double fl = orc_wave_fn(ps, &L, gamma, &dl);
    double fr = orc_wave_fn(ps, &R, gamma, &dr);
    double us = 0.5 * (ul + ur) + 0.5 * (fr - fl);
    double g1 = (gamma - 1.0) / (gamma + 1.0);
    double rsl, rsr;
    if (ps > pl) rsl = rl * (ps / pl + g1) / (g1 * ps / pl + 1.0);
    else rsl = rl * pow(ps / pl, 1.0 / gamma);
    if (ps > pr) rsr = rr * (ps / pr + g1) / (g1 * ps / pr + 1.0);
    else rsr = rr * pow(ps / pr, 1.0 / gamma);
    out[0] = ps; out[1] = us; out[2] = rsl; out[3] = rsr;
    return 0;
}

/* Sample the exact solution at similarity coordinates xi = (x - x0)/t.
 * waves (optional, 5 values): left-wave head, left-wave tail, contact,
 * right-wave tail, right-wave head speeds (shock: head == tail).            */
int orc_riemann_sample(double rl, double ul, double pl, double rr, double ur, double pr,
                       double gamma, const double *xi, int64_t nxi,
                       double *rho, double *u, double *p, double *waves)
{
    double st[4];
    if (orc_riemann_star(rl, ul, pl, rr, ur, pr, gamma, st) != 0) return -1;
    double ps = st[0], us = st[1], rsl = st[2], rsr = st[3];
    double cl = sqrt(gamma * pl / rl), cr = sqrt(gamma * pr / rr);
    double gp = (gamma + 1.0) / (2.0 * gamma), gm = (gamma - 1.0) / (2.0 * gamma);
    double hl, tl, hr, tr;
    if (ps > pl) { hl = tl = ul - cl * sqrt(gp * ps / pl + gm); }
    else { hl = ul - cl; tl = us - cl * pow(ps / pl, gm); }
    if (ps > pr) { hr = tr = ur + cr * sqrt(gp * ps / pr + gm); }
    else { hr = ur + cr; tr = us + cr * pow(ps / pr, gm); }
    if (waves) { waves[0] = hl; waves[1] = tl; waves[2] = us; waves[3] = tr; waves[4] = hr; }
    double g2 = 2.0 / (gamma + 1.0), g3 = (gamma - 1.0) / (gamma + 1.0);
    for (int64_t i = 0; i < nxi; ++i) {
        double s = xi[i];
        double R_, U_, P_;
        if (s <= us) {
            if (s <= hl) { R_ = rl; U_ = ul; P_ = pl; }
            else if (s >= tl) { R_ = rsl; U_ = us; P_ = ps; }
            else {
                double b = g2 + g3 / cl * (ul - s);
                R_ = rl * pow(b, 2.0 / (gamma - 1.0));
                U_ = g2 * (cl + 0.5 * (gamma - 1.0) * ul + s);
                P_ = pl * pow(b, 2.0 * gamma / (gamma - 1.0));
            }
        } else {
            if (s >= hr) { R_ = rr; U_ = ur; P_ = pr; }
            else if (s <= tr) { R_ = rsr; U_ = us; P_ = ps; }
            else {
                double b = g2 - g3 / cr * (ur - s);
                R_ = rr * pow(b, 2.0 / (gamma - 1.0));
                U_ = g2 * (-cr + 0.5 * (gamma - 1.0) * ur + s);
                P_ = pr * pow(b, 2.0 * gamma / (gamma - 1.0));
            }
        }
        rho[i] = R_; u[i] = U_; p[i] = P_;
    }
    return 0;
}
