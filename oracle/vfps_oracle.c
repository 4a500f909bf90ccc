/*
 * vfps_oracle.c -- plain, slow FP64 CPU oracle for one time step of the
 * normalised Vlasov-Fokker-Planck solver of Schoenfeldt et al.,
 * "A Parallelized Vlasov-Fokker-Planck-Solver for Desktop PCs" (Inovesa).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header or table with the CUDA path.
 *
 * Every routine follows the paper's notation and the order of its steps:
 *   - grid and coordinate transformation            (Sec. III.A, Eq. coordinate trafo)
 *   - Lagrange interpolation on N_I nodes            (Sec. III.A, Eqs. interpolation,
 *                                                      lagrange-basis-polynomials)
 *   - clamped interpolation                          (Sec. III.A, Eq. clamping)
 *   - time step = rotation, kick, damping/diffusion  (Sec. III.B, f = f_rot+f_kick+f_damp,diff)
 *   - Manhattan rotation: energy-dependent drift, then location-dependent
 *     RF kick, each a 1-D interpolation          (Sec. III.B, symplectic rotation)
 *   - wake potential from the impedance              (Sec. II.B, Eq. wakepotential)
 *   - cubic first derivative for the FP term         (Sec. III.B, Eq. cubic diff)
 *   - CSR power P ~ int Re(Z) |rho~|^2 dk            (Sec. IV.C)
 * Readings where the paper is silent or garbled (grid nodes, time units,
 * kick normalisation, FFT length, clamp form, renormalisation) are listed in
 * the design notes; each is restated at the routine that uses it.
 *
 * Everything is double precision.  OpenMP only splits loops whose iterations
 * are independent, so results do not depend on the thread count.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct or_params {
    int n;                 /* grid points per axis                               */
    int steps_per_period;  /* time steps per synchrotron period                  */
    int interp_points;     /* N_I: 2, 3 or 4 (cubic)                             */
    int clamp;             /* 1: clamped interpolation (Eq. clamping)            */
    int fp_derivative;     /* 1: cubic derivative (Eq. cubic diff), 0: central   */
    int pad_factor;        /* FFT length M = pad_factor * n                      */
    int renormalize;       /* 1: rescale the charge to 1 after every step        */
    int rotation;          /* 0: standard rotation, 1: Manhattan rotation        */
    double half_width;     /* L: q, p in [-L, L]                                 */
    double beta;           /* 1 / (f_s tau_d)                                    */
    double s_csr;          /* collective kick strength                           */
} or_params;

/* Grid spacing: nodes q_x = -L + x*Delta, x = 0..n-1 (symmetric grid). */
static double grid_delta(const or_params* pr) { return 2.0 * pr->half_width / (pr->n - 1); }

/* Rotation angle of one time step: one synchrotron period is one full turn. */
static double step_angle(const or_params* pr) { return 2.0 * M_PI / pr->steps_per_period; }

/* FFT length: the smallest power of two >= pad_factor * n (zero padding;
 * equal to pad_factor * n whenever n is a power of two). */
int or_fft_length(const or_params* pr)
{
    int m = 1;
    while (m < pr->pad_factor * pr->n) m <<= 1;
    return m;
}

/* Offset of the first interpolation node from m = floor(m_r): the nodes are
 * m - floor((N_I-1)/2) ... m + ceil((N_I-1)/2)  (Sec. III.A). */
int or_first_node(int ni) { return -((ni - 1) / 2); }

/* Lagrange basis polynomials l_{nu,N}({m}) on the integer node offsets
 * m_k = first + k, evaluated at the fractional part t (Eq.
 * lagrange-basis-polynomials), written as the literal product. */
void or_lagrange(int ni, double t, double* w)
{
    int first = or_first_node(ni);
    for (int nu = 0; nu < ni; ++nu) {
        double l = 1.0;
        for (int k = 0; k < ni; ++k) {
            if (k == nu) continue;
            l *= (t - (double)(first + k)) / (double)(nu - k);
        }
        w[nu] = l;
    }
}

/* psi value at integer node (x, y); zero off the grid. */
static double node(const double* psi, int n, int x, int y)
{
    if (x < 0 || x >= n || y < 0 || y >= n) return 0.0;
    return psi[(size_t)x * n + y];
}

/* A source coordinate more than one cell outside the grid contributes 0. */
static int outside(double r, int n) { return r < -1.0 || r > (double)n; }

static double clamp_to(double v, double a, double b)
{
    double lo = a < b ? a : b, hi = a < b ? b : a;
    if (v < lo) return lo;
    if (v > hi) return hi;
    return v;
}

/* 2-D interpolation of psi at the real grid coordinate (x_r, y_r) with the
 * tensor product of the 1-D Lagrange weights.  With clamping, the result is
 * restricted to [min, max] of the 2x2 nearest nodes. */
double or_interp2(const or_params* pr, const double* psi, double xr, double yr)
{
    int n = pr->n, ni = pr->interp_points;
    if (outside(xr, n) || outside(yr, n)) return 0.0;
    double mxf = floor(xr), myf = floor(yr);
    int mx = (int)mxf, my = (int)myf;
    double wx[4], wy[4];
    or_lagrange(ni, xr - mxf, wx);
    or_lagrange(ni, yr - myf, wy);
    int f0 = or_first_node(ni);
    double v = 0.0;
    for (int a = 0; a < ni; ++a)
        for (int b = 0; b < ni; ++b)
            v += wx[a] * wy[b] * node(psi, n, mx + f0 + a, my + f0 + b);
    if (pr->clamp) {
        double c00 = node(psi, n, mx, my), c10 = node(psi, n, mx + 1, my);
        double c01 = node(psi, n, mx, my + 1), c11 = node(psi, n, mx + 1, my + 1);
        double lo = fmin(fmin(c00, c10), fmin(c01, c11));
        double hi = fmax(fmax(c00, c10), fmax(c01, c11));
        v = clamp_to(v, lo, hi);
    }
    return v;
}

/* 1-D interpolation along p (the contiguous axis) of column x at y_r;
 * clamping restricts to the two nearest nodes (Eq. clamping). */
double or_interp_p(const or_params* pr, const double* psi, int x, double yr)
{
    int n = pr->n, ni = pr->interp_points;
    if (outside(yr, n)) return 0.0;
    double myf = floor(yr);
    int my = (int)myf;
    double w[4];
    or_lagrange(ni, yr - myf, w);
    int f0 = or_first_node(ni);
    double v = 0.0;
    for (int b = 0; b < ni; ++b) v += w[b] * node(psi, n, x, my + f0 + b);
    if (pr->clamp) v = clamp_to(v, node(psi, n, x, my), node(psi, n, x, my + 1));
    return v;
}

/* 1-D interpolation along q of row y at x_r (the drift of the Manhattan
 * rotation); clamping restricts to the two nearest nodes (Eq. clamping). */
double or_interp_q(const or_params* pr, const double* psi, double xr, int y)
{
    int n = pr->n, ni = pr->interp_points;
    if (outside(xr, n)) return 0.0;
    double mxf = floor(xr);
    int mx = (int)mxf;
    double w[4];
    or_lagrange(ni, xr - mxf, w);
    int f0 = or_first_node(ni);
    double v = 0.0;
    for (int a = 0; a < ni; ++a) v += w[a] * node(psi, n, mx + f0 + a, y);
    if (pr->clamp) v = clamp_to(v, node(psi, n, mx, y), node(psi, n, mx + 1, y));
    return v;
}

/* Step parameter h of the Manhattan rotation.  The drift-kick map
 * (q, p) -> (q + h p, p - h (q + h p)) has determinant 1 and trace 2 - h^2,
 * i.e. it turns phase space by mu with 2 cos(mu) = 2 - h^2.  The paper does
 * not state h; h = 2 sin(pi/steps_per_period) makes mu = 2 pi/steps, so that
 * one synchrotron period is again exactly one turn. */
double or_manhattan_h(const or_params* pr) { return 2.0 * sin(M_PI / pr->steps_per_period); }

/* Manhattan rotation, first half (Sec. III.B, symplectic integrator): the
 * energy-dependent drift q -> q + h p moves every row p along q, so the new
 * value at (q, p) is the old one at (q - h p, p). */
void or_drift(const or_params* pr, const double* in, double* out)
{
    int n = pr->n;
    double d = grid_delta(pr), L = pr->half_width, h = or_manhattan_h(pr);
#pragma omp parallel for schedule(static)
    for (int x = 0; x < n; ++x) {
        double q = -L + x * d;
        for (int y = 0; y < n; ++y) {
            double p = -L + y * d;
            out[(size_t)x * n + y] = or_interp_q(pr, in, (q - h * p + L) / d, y);
        }
    }
}

/* Manhattan rotation, second half: the location-dependent RF kick
 * p -> p - h q moves every column q along p, so the new value at (q, p) is
 * the old one at (q, p + h q). */
void or_rfkick(const or_params* pr, const double* in, double* out)
{
    int n = pr->n;
    double d = grid_delta(pr), L = pr->half_width, h = or_manhattan_h(pr);
#pragma omp parallel for schedule(static)
    for (int x = 0; x < n; ++x) {
        double q = -L + x * d;
        for (int y = 0; y < n; ++y) {
            double p = -L + y * d;
            out[(size_t)x * n + y] = or_interp_p(pr, in, x, (p + h * q + L) / d);
        }
    }
}

/* RotationMap ("standard rotation", Sec. III.B): the new value at (q, p) is
 * the old density at the point that the unperturbed flow dq/dtheta = p,
 * dp/dtheta = -q carries onto (q, p) in one step, i.e. rotated back by the
 * step angle.  Coordinates use the transformation y_r = (p - p_min)/Delta p. */
void or_rotate(const or_params* pr, const double* in, double* out)
{
    int n = pr->n;
    double d = grid_delta(pr), L = pr->half_width, phi = step_angle(pr);
    double cs = cos(phi), sn = sin(phi);
#pragma omp parallel for schedule(static)
    for (int x = 0; x < n; ++x) {
        double q = -L + x * d;
        for (int y = 0; y < n; ++y) {
            double p = -L + y * d;
            double qs = q * cs - p * sn;
            double ps = q * sn + p * cs;
            double xr = (qs + L) / d, yr = (ps + L) / d;
            out[(size_t)x * n + y] = or_interp2(pr, in, xr, yr);
        }
    }
}

/* Bunch profile rho(q) = int psi dp, rectangle rule; returns the charge
 * Q = int rho dq (Sec. II.B: the profile whose transform enters the wake). */
double or_project(const or_params* pr, const double* psi, double* rho)
{
    int n = pr->n;
    double d = grid_delta(pr);
    double q = 0.0;
    for (int x = 0; x < n; ++x) {
        double s = 0.0;
        for (int y = 0; y < n; ++y) s += psi[(size_t)x * n + y];
        rho[x] = d * s;
        q += d * rho[x];
    }
    return q;
}

/* Wake potential and CSR power (Eq. wakepotential, Sec. IV.C).
 *   rho~_k = Delta * sum_{i<n} rho_i exp(-2 pi i ik/M),      k = 0..M/2,
 *   V_l    = 2 dkappa Re sum_{k=1}^{M/2-1} Z_k rho~_k exp(+2 pi i lk/M),
 *   P      = dkappa sum_{k=1}^{M/2-1} 2 Re(Z_k) |rho~_k|^2,
 * with M >= pad*n a power of two (zero padding), kappa_k = k dkappa,
 * dkappa = 2 pi/(M Delta).
 * The kappa < 0 half follows from Hermitian symmetry; the DC term vanishes
 * because Z(0) = 0 and the Nyquist bin is dropped.  This is the direct DFT
 * of the definition, O(n M), with no fast transform. */
void or_wake(const or_params* pr, const double* zre, const double* zim,
             const double* rho, double* V, double* P)
{
    int n = pr->n, M = or_fft_length(pr), K = M / 2;
    double d = grid_delta(pr), dk = 2.0 * M_PI / (M * d);
    double* ct = (double*)malloc(sizeof(double) * M);
    double* st = (double*)malloc(sizeof(double) * M);
    double* rr = (double*)malloc(sizeof(double) * (K + 1));
    double* ri = (double*)malloc(sizeof(double) * (K + 1));
    for (int m = 0; m < M; ++m) {
        ct[m] = cos(2.0 * M_PI * m / M);
        st[m] = sin(2.0 * M_PI * m / M);
    }
#pragma omp parallel for schedule(static)
    for (int k = 0; k <= K; ++k) {
        double re = 0.0, im = 0.0;
        for (int i = 0; i < n; ++i) {
            int m = (int)(((long long)i * k) % M);
            re += rho[i] * ct[m];
            im -= rho[i] * st[m];
        }
        rr[k] = d * re;
        ri[k] = d * im;
    }
#pragma omp parallel for schedule(static)
    for (int l = 0; l < n; ++l) {
        double s = 0.0;
        for (int k = 1; k < K; ++k) {
            int m = (int)(((long long)l * k) % M);
            /* Re[(zr + i zi)(rr + i ri)(c + i s)] */
            double ar = zre[k] * rr[k] - zim[k] * ri[k];
            double ai = zre[k] * ri[k] + zim[k] * rr[k];
            s += ar * ct[m] - ai * st[m];
        }
        V[l] = 2.0 * dk * s;
    }
    if (P) {
        double s = 0.0;
        for (int k = 1; k < K; ++k) s += 2.0 * zre[k] * (rr[k] * rr[k] + ri[k] * ri[k]);
        *P = dk * s;
    }
    free(ct); free(st); free(rr); free(ri);
}

/* WakeKickMap (Sec. III.B): the wake is turned into a kick along p,
 * dp = +S_csr * V(q) * phi over one step of phi radians, and translated to
 * grid units with the coordinate transformation, y_r = y - dp/Delta p.  Each
 * column q_x is shifted along p by its own amount with 1-D interpolation.
 * Sign: with the printed transform V = int Z rho~ e^{ikq} dk the CSR kernel
 * acts toward +q, so +q is the bunch head; the printed Hamiltonian's flow
 * dq/dtheta = p then makes p grow as the energy falls (above transition), and
 * the energy lost to the wake raises p.  This reading gives the free-space
 * threshold S_csr ~ 0.5 that the paper quotes (Sec. IV.B). */
void or_kick(const or_params* pr, const double* V, const double* in, double* out)
{
    int n = pr->n;
    double d = grid_delta(pr), phi = step_angle(pr);
#pragma omp parallel for schedule(static)
    for (int x = 0; x < n; ++x) {
        double dp = pr->s_csr * V[x] * phi;
        for (int y = 0; y < n; ++y)
            out[(size_t)x * n + y] = or_interp_p(pr, in, x, (double)y - dp / d);
    }
}

/* FokkerPlanckMap: one explicit Euler step of the right-hand side of Eq. VFP,
 * beta d/dp (p psi + d psi/dp) = beta (psi + p psi' + psi''), over a time step
 * of 1/steps_per_period synchrotron periods.  psi' is the cubic derivative of
 * Eq. cubic diff (or the central difference), psi'' the three-point second
 * difference; values off the grid are zero. */
void or_fokker_planck(const or_params* pr, const double* in, double* out)
{
    int n = pr->n;
    double d = grid_delta(pr), L = pr->half_width;
    double h = pr->beta / pr->steps_per_period;
#pragma omp parallel for schedule(static)
    for (int x = 0; x < n; ++x) {
        for (int y = 0; y < n; ++y) {
            double p = -L + y * d;
            double fm = node(in, n, x, y - 1), f0 = node(in, n, x, y);
            double fp = node(in, n, x, y + 1), fpp = node(in, n, x, y + 2);
            double d1;
            if (pr->fp_derivative)
                d1 = (-2.0 * fm - 3.0 * f0 + 6.0 * fp - fpp) / (6.0 * d);
            else
                d1 = (fp - fm) / (2.0 * d);
            double d2 = (fp - 2.0 * f0 + fm) / (d * d);
            out[(size_t)x * n + y] = f0 + h * (f0 + p * d1 + d2);
        }
    }
}

/* Bunch moments of psi (first and second moments of the distribution in q
 * and p, the quantities behind the paper's bunch length and energy spread):
 * out = {<q>, sigma_q, <p>, sigma_p} with <f> = sum f psi / sum psi over the
 * nodes, sigma^2 = <f^2> - <f>^2. */
void or_moments(const or_params* pr, const double* psi, double* out)
{
    int n = pr->n;
    double d = grid_delta(pr), L = pr->half_width;
    double s0 = 0.0, sq = 0.0, sqq = 0.0, sp = 0.0, spp = 0.0;
    for (int x = 0; x < n; ++x) {
        double q = -L + x * d;
        for (int y = 0; y < n; ++y) {
            double p = -L + y * d, v = psi[(size_t)x * n + y];
            s0 += v;
            sq += q * v;
            sqq += q * q * v;
            sp += p * v;
            spp += p * p * v;
        }
    }
    double mq = sq / s0, mp = sp / s0;
    out[0] = mq;
    out[1] = sqrt(sqq / s0 - mq * mq);
    out[2] = mp;
    out[3] = sqrt(spp / s0 - mp * mp);
}

/* Charge Q = Delta^2 sum psi. */
double or_charge(const or_params* pr, const double* psi)
{
    size_t nn = (size_t)pr->n * pr->n;
    double d = grid_delta(pr), s = 0.0;
    for (size_t i = 0; i < nn; ++i) s += psi[i];
    return d * d * s;
}

/* Scale psi so that its charge is 1; returns the charge before scaling. */
double or_normalize(const or_params* pr, double* psi)
{
    size_t nn = (size_t)pr->n * pr->n;
    double q = or_charge(pr, psi);
    for (size_t i = 0; i < nn; ++i) psi[i] /= q;
    return q;
}

/* One time step, in the order
 *   1. profile and charge of psi_t,  2. wake and CSR power,  3. rotation
 *   (standard, or Manhattan: drift then RF kick),  4. kick,  5. damping and
 *   diffusion,  6. renormalisation to charge 1.
 * The collective force is held fixed over the step (Sec. II.A).
 * work must hold 2*n*n doubles.  Outputs (any may be NULL): rho and V of
 * psi_t (n each), P of psi_t, and the charge before renormalisation. */
void or_step(const or_params* pr, const double* zre, const double* zim,
             double* psi, double* work, double* rho_out, double* V_out,
             double* P_out, double* Qpre_out)
{
    int n = pr->n;
    size_t nn = (size_t)n * n;
    double* rho = (double*)malloc(sizeof(double) * n);
    double* V = (double*)malloc(sizeof(double) * n);
    double* a = work;
    double* b = work + nn;
    double P = 0.0;
    or_project(pr, psi, rho);
    or_wake(pr, zre, zim, rho, V, &P);
    if (pr->rotation == 1) {
        or_drift(pr, psi, a);
        or_rfkick(pr, a, b);
        or_kick(pr, V, b, a);
        or_fokker_planck(pr, a, psi);
    } else {
        or_rotate(pr, psi, a);
        or_kick(pr, V, a, b);
        or_fokker_planck(pr, b, psi);
    }
    double q = or_charge(pr, psi);
    if (pr->renormalize)
        for (size_t i = 0; i < nn; ++i) psi[i] /= q;
    if (rho_out) memcpy(rho_out, rho, sizeof(double) * n);
    if (V_out) memcpy(V_out, V, sizeof(double) * n);
    if (P_out) *P_out = P;
    if (Qpre_out) *Qpre_out = q;
    free(rho); free(V);
}

/* nsteps consecutive steps; P_series[t] and Q_series[t] (may be NULL) get the
 * CSR power of psi_t and the charge before renormalisation of step t. */
void or_run(const or_params* pr, const double* zre, const double* zim,
            double* psi, long long nsteps, double* P_series, double* Q_series)
{
    size_t nn = (size_t)pr->n * pr->n;
    double* work = (double*)malloc(sizeof(double) * 2 * nn);
    for (long long t = 0; t < nsteps; ++t) {
        double P, Q;
        or_step(pr, zre, zim, psi, work, NULL, NULL, &P, &Q);
        if (P_series) P_series[t] = P;
        if (Q_series) Q_series[t] = Q;
    }
    free(work);
}

/* Power spectrum of a CSR-power series (the rows of the paper's bursting
 * spectrogram, Sec. IV.C): the last L values x_j of the series, their mean
 * removed, times the Hann window h_j = (1 - cos(2 pi j/L))/2, and
 * out[k] = |sum_j h_j (x_j - mean) exp(-2 pi i j k/L)|^2 for k = 0..L/2,
 * written as the direct sum.  Frequency k is k steps_per_period/L cycles per
 * synchrotron period. */
void or_power_spectrum(const double* x, int L, double* out)
{
    double mean = 0.0;
    for (int j = 0; j < L; ++j) mean += x[j];
    mean /= L;
#pragma omp parallel for schedule(static)
    for (int k = 0; k <= L / 2; ++k) {
        double re = 0.0, im = 0.0;
        for (int j = 0; j < L; ++j) {
            double h = 0.5 * (1.0 - cos(2.0 * M_PI * j / L));
            double a = -2.0 * M_PI * (double)j * (double)k / L;
            re += h * (x[j] - mean) * cos(a);
            im += h * (x[j] - mean) * sin(a);
        }
        out[k] = re * re + im * im;
    }
}
