/*
 * qr_oracle.c -- plain FP64 CPU oracle of the QRMC scheme (arXiv 2407.21084).
 *
 * TEST INFRASTRUCTURE ONLY (see qr_oracle.h). Slow on purpose: every step is
 * written the way the paper states it, with no blocking, fusion or
 * reordering beyond the definitions, so that it can be checked by eye:
 *
 *   Euler scheme            Sec. 2.1.1, eq. (alg:markov:euler)
 *   random start X_i^i ~ nu Sec. 2.1.2, assumption (H_nu): product density,
 *                           inverse-CDF sampling per coordinate (Sec. 5)
 *   basis                   Sec. 2.2, tensor products of 1-D functions of
 *                           F_nu(x_l) (eq. phi:dim:d, relation:1): either the
 *                           complex exponentials e^{2 pi i k u}, k in Z, which
 *                           are orthonormal on [0,1] exactly as the cosines
 *                           of Lemma (ortho:dim1), or (basis = 1) the cosines
 *                           C_0 = 1, C_k = sqrt(2) cos(k pi u), k in N, of
 *                           Lemma (ortho:dim1) itself; Lemma (eqInnerNorms)
 *                           makes phi_k orthonormal in L2_nu in both cases.
 *   response S_i            Sec. 2.3, Algorithm 1, eq. (Sqi:bar:M), damping
 *                           exponent q of eq. (yqi) (q = 0: no weight)
 *   truncation T_L          Sec. 1 notation, eq. (TL:2), constant L
 *   coefficients            Sec. 2.3, Algorithm 1, eq. (Aqi:bar:M): plain
 *                           Monte-Carlo average, no linear solve
 *   Picard iteration        all i at once from the previous iterate (Jacobi);
 *                           Algorithm 1's backward sweep is ora_backward_sweep
 */
#include "qr_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ Gamma */

static int gamma_partial_ok(int kind, int n, const int* k, int upto)
{
    /* Feasibility of the prefix k[0..upto]: the remaining coordinates can
     * always be 0, which adds 0 to the l1 sum and 1 to the product. */
    long long s = 0, prod = 1;
    for (int l = 0; l <= upto; ++l) {
        int a = k[l] < 0 ? -k[l] : k[l];
        switch (kind) {
        case ORA_G_LINF_Z:
        case ORA_G_FULL_N:
            if (a > n) return 0;
            break;
        case ORA_G_L1_Z:
        case ORA_G_TOTAL_N:
            s += a;
            if (s > n) return 0;
            break;
        case ORA_G_HYP_Z:
        case ORA_G_HYP_N:
            prod *= (a > 1 ? a : 1);
            if (prod > n) return 0;
            break;
        default:
            return 0;
        }
    }
    return 1;
}

static long long gamma_rec(int kind, int d, int n, int l, int* k, int* k_out, long long cap,
                           long long count)
{
    int is_z = (kind == ORA_G_LINF_Z || kind == ORA_G_L1_Z || kind == ORA_G_HYP_Z);
    int lo = is_z ? -n : 0;
    for (int v = lo; v <= n; ++v) {
        k[l] = v;
        if (!gamma_partial_ok(kind, n, k, l)) continue;
        if (l == d - 1) {
            if (k_out && count < cap) memcpy(k_out + count * d, k, sizeof(int) * (size_t)d);
            ++count;
        } else {
            count = gamma_rec(kind, d, n, l + 1, k, k_out, cap, count);
        }
    }
    return count;
}

long long ora_gamma_list(int kind, int d, int n, int* k_out, long long cap)
{
    if (d < 1 || d > 32 || n < 0 || kind < 0 || kind > ORA_G_HYP_N) return -1;
    if ((kind == ORA_G_HYP_Z || kind == ORA_G_HYP_N) && n < 1) return -1;
    int k[32];
    return gamma_rec(kind, d, n, 0, k, k_out, cap, 0);
}

long long ora_gamma_count(int kind, int d, int n) { return ora_gamma_list(kind, d, n, NULL, 0); }

/* ----------------------------------------------------------------- Philox */

void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    /* Salmon et al. (SC'11), Philox4x32 with 10 rounds: each round multiplies
     * words 0 and 2 by the two Philox constants, and the key is bumped by the
     * Weyl constants between rounds. */
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

double ora_u01(uint32_t a, uint32_t b)
{
    uint64_t n = ((uint64_t)a << 20) ^ (uint64_t)(b >> 12); /* 52 bits */
    return (double)(2 * n + 1) * 0x1p-53;
}

static void philox_call(uint64_t seed, int instance, int tag, int i, uint32_t m, uint32_t c,
                        uint32_t j, uint32_t out[4])
{
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {m, c, j, ((uint32_t)instance << 20) | ((uint32_t)tag << 16) | (uint32_t)i};
    ora_philox4x32_10(ctr, key, out);
}

void ora_start_uniforms(uint64_t seed, int instance, int i, uint32_t m, int d, double* u)
{
    for (int c = 0; 2 * c < d; ++c) {
        uint32_t r[4];
        philox_call(seed, instance, ORA_TAG_START, i, m, (uint32_t)c, 0xffffffffu, r);
        u[2 * c] = ora_u01(r[0], r[1]);
        if (2 * c + 1 < d) u[2 * c + 1] = ora_u01(r[2], r[3]);
    }
}

void ora_test_uniforms(uint64_t seed, int instance, int i, uint32_t p, int d, double* u)
{
    for (int c = 0; 2 * c < d; ++c) {
        uint32_t r[4];
        philox_call(seed, instance, ORA_TAG_TEST, i, p, (uint32_t)c, 0xffffffffu, r);
        u[2 * c] = ora_u01(r[0], r[1]);
        if (2 * c + 1 < d) u[2 * c + 1] = ora_u01(r[2], r[3]);
    }
}

void ora_normals(uint64_t seed, int instance, int i, uint32_t m, int j, int d, double* z)
{
    /* Box-Muller on the two uniforms of one Philox call. */
    for (int c = 0; 2 * c < d; ++c) {
        uint32_t r[4];
        philox_call(seed, instance, ORA_TAG_INCR, i, m, (uint32_t)c, (uint32_t)j, r);
        double ua = ora_u01(r[0], r[1]);
        double ub = ora_u01(r[2], r[3]);
        double rho = sqrt(-2.0 * log(ua));
        z[2 * c] = rho * cos(2.0 * M_PI * ub);
        if (2 * c + 1 < d) z[2 * c + 1] = rho * sin(2.0 * M_PI * ub);
    }
}

/* -------------------------------------------------------------------- nu */

double ora_nu_pdf(int kind, double mu, double x)
{
    switch (kind) {
    case ORA_NU_LOMAX:
        return 0.5 * mu * pow(1.0 + fabs(x), -(mu + 1.0));
    case ORA_NU_STUDENT2:
        return 0.5 * pow(1.0 + x * x, -1.5);
    case ORA_NU_CAUCHY:
        return 1.0 / (M_PI * (1.0 + x * x));
    }
    return NAN;
}

double ora_nu_cdf(int kind, double mu, double x)
{
    switch (kind) {
    case ORA_NU_LOMAX:
        return x < 0 ? 0.5 * pow(1.0 + fabs(x), -mu) : 1.0 - 0.5 * pow(1.0 + x, -mu);
    case ORA_NU_STUDENT2: /* Sec. 5, eq. (Fnui:Fnulinv) */
        return 0.5 * (x / sqrt(x * x + 1.0) + 1.0);
    case ORA_NU_CAUCHY:
        return 0.5 + atan(x) / M_PI;
    }
    return NAN;
}

double ora_nu_icdf(int kind, double mu, double u)
{
    switch (kind) {
    case ORA_NU_LOMAX: {
        double w = u < 0.5 ? u : 1.0 - u;
        double x = pow(2.0 * w, -1.0 / mu) - 1.0;
        return u < 0.5 ? -x : x;
    }
    case ORA_NU_STUDENT2: { /* Sec. 5, eq. (Fnui:Fnulinv) */
        double r = sqrt((-u * u + u - 0.25) / (u * (u - 1.0)));
        return u <= 0.5 ? -r : r;
    }
    case ORA_NU_CAUCHY: /* Sec. 5 (mixed smoothness): tan(pi u - pi/2) */
        return tan(M_PI * u - 0.5 * M_PI);
    }
    return NAN;
}

/* ----------------------------------------------------------- f, g, series */

static int gamma_kmax(const ora_problem* p)
{
    if (p->kmax > 0) return p->kmax;
    int K = 0;
    for (long long e = 0; e < (long long)p->nG * p->d; ++e) {
        int a = p->k[e] < 0 ? -p->k[e] : p->k[e];
        if (a > K) K = a;
    }
    return K;
}

/* 1-D factors of phi_k at u[0..d-1] (Sec. 2.2), E[l][v+K] for v = -K..K:
 * e^{2 pi i v u_l} for the Fourier basis; for the cosine basis of Lemma
 * (ortho:dim1) C_v(u_l) = 1 (v = 0), sqrt(2) cos(v pi u_l) (v > 0), real
 * (entries with v < 0 are never used: the cosine sets lie in N^d). */
static void factor_table(const ora_problem* p, const double* u, int K, double complex* E)
{
    int W = 2 * K + 1;
    for (int l = 0; l < p->d; ++l)
        for (int v = -K; v <= K; ++v) {
            if (p->basis == ORA_BASIS_COS) {
                E[l * W + v + K] = v == 0 ? 1.0 : (v > 0 ? sqrt(2.0) * cos(M_PI * (double)v * u[l]) : 0.0);
            } else {
                double th = 2.0 * M_PI * (double)v * u[l];
                E[l * W + v + K] = cos(th) + I * sin(th);
            }
        }
}

/* Series y = Re sum_k alpha_k phi_k at the point whose images under F_nu
 * are u[0..d-1] (for the cosine basis phi_k and alpha_k are real). */
static double series_at_u(const ora_problem* p, const double* alpha, const double* u)
{
    int d = p->d, K = gamma_kmax(p), W = 2 * K + 1;
    double complex E[d * W];
    factor_table(p, u, K, E);
    double complex y = 0;
    for (int e = 0; e < p->nG; ++e) {
        double complex phi = 1.0;
        for (int l = 0; l < d; ++l) phi *= E[l * W + p->k[e * d + l] + K];
        y += (alpha[2 * e] + I * alpha[2 * e + 1]) * phi;
    }
    return creal(y);
}

double ora_series(const ora_problem* p, const double* alpha, const double* x)
{
    double u[32];
    for (int l = 0; l < p->d; ++l) u[l] = ora_nu_cdf(p->nu_kind, p->mu, x[l]);
    return series_at_u(p, alpha, u);
}

static double dot_s_x(const double* s, const double* x, int d)
{
    double a = 0;
    for (int l = 0; l < d; ++l) a += s[l] * x[l];
    return a;
}

double ora_g(const ora_problem* p, const double* x)
{
    int d = p->d;
    switch (p->g_kind) {
    case ORA_GT_COS:
        return cos(dot_s_x(p->g_par, x, d));
    case ORA_GT_TRIGPOLY:
        return ora_series(p, p->g_par, x);
    case ORA_GT_PAPER_SIN: { /* Sec. 5: g = 1 + kappa + sin(lambda sum x_l) */
        double sx = 0;
        for (int l = 0; l < d; ++l) sx += x[l];
        return 1.0 + p->g_par[0] + sin(p->g_par[1] * sx);
    }
    }
    return NAN;
}

double ora_f(const ora_problem* p, double t, const double* x, double y)
{
    int d = p->d;
    switch (p->f_kind) {
    case ORA_F_ZERO:
        return 0.0;
    case ORA_F_LINEAR:
        return p->f_par[0] * y;
    case ORA_F_CUBIC_MANUF: {
        /* u = e^{a(T-t)} cos(s.x) solves d_t u + (1/2) tr(sigma sigma^T D^2 u)
         * + f(t,x,u) = 0 for f = -y^3 + r, r = (a + |sigma^T s|^2/2) u + u^3. */
        double a = p->f_par[0];
        const double* s = p->f_par + 1;
        double st2 = 0;
        for (int c = 0; c < d; ++c) {
            double v = 0;
            for (int l = 0; l < d; ++l) v += p->sigma[l * d + c] * s[l];
            st2 += v * v;
        }
        double u = exp(a * (p->T - t)) * cos(dot_s_x(s, x, d));
        double r = (a + 0.5 * st2) * u + u * u * u;
        return -y * y * y + r;
    }
    case ORA_F_PAPER_MIN: { /* Sec. 5 */
        double kap = p->f_par[0], lam = p->f_par[1], sx = 0;
        for (int l = 0; l < d; ++l) sx += x[l];
        double v = y - kap - 1.0 - sin(lam * sx) * exp(lam * lam * (double)d * (t - p->T) / 2.0);
        v = v * v;
        return v < 1.0 ? v : 1.0;
    }
    }
    return NAN;
}

/* ------------------------------------------------------------- the scheme */

static void start_point(const ora_problem* p, int i, long long m, double* u)
{
    if (p->lattice_n > 0) {
        long long r = m;
        for (int l = 0; l < p->d; ++l) {
            u[l] = ((double)(r % p->lattice_n) + 0.5) / (double)p->lattice_n;
            r /= p->lattice_n;
        }
    } else {
        ora_start_uniforms(p->seed, p->instance, i, (uint32_t)m, p->d, u);
    }
}

/* Damping weight (1 + |x|^2)^{q/2} of eq. (yqi). */
static double damp_weight(const ora_problem* p, const double* x)
{
    double r2 = 0;
    for (int l = 0; l < p->d; ++l) r2 += x[l] * x[l];
    return pow(1.0 + r2, 0.5 * p->q_damp);
}

double ora_response(const ora_problem* p, const double* alpha, int i, long long m, double* u_out,
                    long long* clamp_hits)
{
    int d = p->d, N = p->N;
    double dt = p->T / (double)N, sq = sqrt(dt);
    double x[32], x1[32], z[32];
    start_point(p, i, m, u_out);
    for (int l = 0; l < d; ++l) x[l] = ora_nu_icdf(p->nu_kind, p->mu, u_out[l]); /* X_i^i ~ nu */
    double w_start = p->q_damp != 0.0 ? damp_weight(p, x) : 1.0;
    double sum_f = 0.0;
    for (int j = i; j < N; ++j) {
        /* Euler step: X_{j+1} = X_j + b dt + sigma (W_{t_{j+1}} - W_{t_j}) */
        ora_normals(p->seed, p->instance, i, (uint32_t)m, j, d, z);
        for (int l = 0; l < d; ++l) {
            double noise = 0;
            for (int c = 0; c < d; ++c) noise += p->sigma[l * d + c] * z[c];
            x1[l] = x[l] + p->b[l] * dt + noise * sq;
        }
        /* y_{j+1}(X_{j+1}): g at the terminal time, else the previous
         * iterate's series, truncated by T_L. */
        double y1;
        if (j + 1 == N) {
            y1 = ora_g(p, x1);
        } else {
            /* the series represents the damped ybar^q_{j+1} (eq. yqi:bar:M):
             * y_{j+1} = ybar^q_{j+1}(X_{j+1}) (1 + |X_{j+1}|^2)^{q/2} */
            y1 = ora_series(p, alpha + (size_t)2 * (size_t)(j + 1) * (size_t)p->nG, x1);
            if (p->q_damp != 0.0) y1 *= damp_weight(p, x1);
            if (p->clamp_L > 0) {
                if (y1 > p->clamp_L) {
                    y1 = p->clamp_L;
                    if (clamp_hits) ++*clamp_hits;
                } else if (y1 < -p->clamp_L) {
                    y1 = -p->clamp_L;
                    if (clamp_hits) ++*clamp_hits;
                }
            }
        }
        sum_f += ora_f(p, (double)j * dt, x, y1) * dt; /* f_j(X_j, y_{j+1}) dt */
        memcpy(x, x1, sizeof(double) * (size_t)d);
    }
    /* S^q_i = [g(X_N) + sum_j f_j(...) dt] / (1 + |X_i^i|^2)^{q/2}, eq. (Sqi:bar:M) */
    double S = ora_g(p, x) + sum_f;
    return p->q_damp != 0.0 ? S / w_start : S;
}

static long long chunk_len(long long len)
{
    long long c = len / 256;
    return c < 1024 ? 1024 : c;
}

/* alpha_i,k = (1/M') sum_{m in [m_lo,m_hi)} S_i^m conj(phi_k(X_i^{i,m})),
 * phi_k evaluated at the exact start uniforms (F_nu(X_i^i) = U); for the
 * real cosine basis conj(phi_k) = phi_k. */
static int project_row(const ora_problem* p, const double* alpha_src, int i, long long m_lo,
                       long long m_hi, double* row_out, long long* clamp_hits)
{
    int d = p->d, nG = p->nG, K = gamma_kmax(p), W = 2 * K + 1;
    long long len = m_hi - m_lo, cl = chunk_len(len);
    long long nch = (len + cl - 1) / cl;
    double complex* part = (double complex*)calloc((size_t)(nch * nG), sizeof(double complex));
    if (!part) return 1;
    long long hits = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : hits)
    for (long long c = 0; c < nch; ++c) {
        double u[32];
        double complex E[d * W];
        double complex* acc = part + c * nG;
        long long a = m_lo + c * cl, bnd = a + cl < m_hi ? a + cl : m_hi;
        for (long long m = a; m < bnd; ++m) {
            long long h = 0;
            double S = ora_response(p, alpha_src, i, m, u, &h);
            hits += h;
            factor_table(p, u, K, E);
            for (int e = 0; e < nG; ++e) {
                double complex phi = 1.0;
                for (int l = 0; l < d; ++l) phi *= E[l * W + p->k[e * d + l] + K];
                acc[e] += S * conj(phi);
            }
        }
    }
    for (int e = 0; e < nG; ++e) {
        double complex s = 0;
        for (long long c = 0; c < nch; ++c) s += part[c * nG + e];
        s /= (double)len;
        row_out[2 * e] = creal(s);
        row_out[2 * e + 1] = cimag(s);
    }
    free(part);
    if (clamp_hits) *clamp_hits += hits;
    return 0;
}

int ora_picard_iter(const ora_problem* p, const double* alpha_in, double* alpha_out, int i_lo,
                    int i_hi, long long m_lo, long long m_hi, int nthreads, long long* clamp_hits)
{
    if (!p || p->d < 1 || p->d > 32 || p->N < 1 || i_lo < 0 || i_hi > p->N || m_hi <= m_lo)
        return 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    (void)nthreads;
    size_t row = (size_t)2 * (size_t)p->nG;
    for (int i = i_lo; i < i_hi; ++i)
        if (project_row(p, alpha_in, i, m_lo, m_hi, alpha_out + row * (size_t)i, clamp_hits))
            return 2;
    return 0;
}

int ora_backward_sweep(const ora_problem* p, double* alpha, long long m_lo, long long m_hi,
                       int nthreads, long long* clamp_hits)
{
    if (!p || p->N < 1 || m_hi <= m_lo) return 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    (void)nthreads;
    size_t row = (size_t)2 * (size_t)p->nG;
    double* tmp = (double*)malloc(sizeof(double) * row);
    for (int i = p->N - 1; i >= 0; --i) {
        if (project_row(p, alpha, i, m_lo, m_hi, tmp, clamp_hits)) {
            free(tmp);
            return 2;
        }
        memcpy(alpha + row * (size_t)i, tmp, sizeof(double) * row);
    }
    free(tmp);
    return 0;
}

int ora_responses(const ora_problem* p, const double* alpha_in, int i, long long m_lo,
                  long long m_hi, double* S_out, int nthreads)
{
    if (!p || i < 0 || i >= p->N || m_hi <= m_lo) return 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    (void)nthreads;
#pragma omp parallel for schedule(static)
    for (long long m = m_lo; m < m_hi; ++m) {
        double u[32];
        S_out[m - m_lo] = ora_response(p, alpha_in, i, m, u, NULL);
    }
    return 0;
}

int ora_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
