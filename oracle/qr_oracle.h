/*
 * qr_oracle.h -- FP64 CPU oracle for the Quasi-Regression Monte-Carlo (QRMC)
 * scheme of Gobet, Lopez-Salas and Vazquez (arXiv 2407.21084).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library. It shares no code,
 * header or table with the CUDA library: the Philox generator, the index-set
 * enumerator, the sampling density and the scheme itself are written here a
 * second time, plainly, in double precision.
 *
 * Parity status per function (pins live in tests/test_oracle_*.py):
 *   ora_gamma_*          pinned: every cardinality printed in Sec. 2.4.2
 *                        (table of #Gamma_T / #Gamma_H) and the result tables
 *                        of Sec. 5, the paper's own counting formula, closed
 *                        forms for the Z^d sets, brute-force membership.
 *   ora_philox4x32_10    pinned: published known-answer vectors of
 *                        Philox4x32-10 (Salmon et al., SC'11).
 *   ora_u01 / normals    pinned: exact bit layout, moments, KS tests.
 *   ora_nu_*             pinned: scipy's Lomax / Student-t / Cauchy laws,
 *                        density normalisation, inverse round trip, KS test.
 *   cosine basis         pinned: planted cosine polynomial recovered exactly
 *                        on a midpoint lattice; sampled orthonormality; the
 *                        paper's d = 1 confidence intervals for u(0,0) = 1.6
 *                        (Sec. 5) on its own test PDE.
 *   damping q            pinned: with sigma = 0 on a lattice the damped
 *                        linear-driver iterate is (1 + lambda dt)^{N-i} times
 *                        the lattice projection of g / w; Feynman-Kac with
 *                        f = 0 against the exact damped coefficients by
 *                        1-D quadrature.
 *   ora_picard_iter      pinned: planted trigonometric polynomial recovered
 *                        exactly on a lattice; the linear driver closed form;
 *                        Feynman-Kac (f=0, drift) against exact coefficients
 *                        from 1-D quadrature; Picard(N) == backward sweep;
 *                        linearity in the path range; manufactured cubic
 *                        solution (statistical, against exact projections).
 */
#ifndef QR_ORACLE_H
#define QR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- index sets Gamma (Sec. 2.4.2 for the N^d sets; Z^d variants for the
 *      complex Fourier basis). Canonical order: lexicographic, k_1 most
 *      significant, integer order on each coordinate. */
enum {
    ORA_G_LINF_Z = 0,  /* {k in Z^d : max|k_l| <= n} */
    ORA_G_L1_Z = 1,    /* {k in Z^d : sum|k_l| <= n} */
    ORA_G_HYP_Z = 2,   /* {k in Z^d : prod max(|k_l|,1) <= n} */
    ORA_G_FULL_N = 3,  /* Gamma_F(n,...,n) = {k in N^d : k_l <= n} */
    ORA_G_TOTAL_N = 4, /* Gamma_T(n) = {k in N^d : sum k_l <= n} */
    ORA_G_HYP_N = 5    /* Gamma_H(n) = {k in N^d : prod max(k_l,1) <= n} */
};
/* Number of elements; -1 on bad arguments. */
long long ora_gamma_count(int kind, int d, int n);
/* Writes |Gamma|*d ints (row per k) in canonical order; returns |Gamma| or -1.
 * k_out may be NULL (count only). cap = capacity of k_out in rows. */
long long ora_gamma_list(int kind, int d, int n, int* k_out, long long cap);

/* ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11). */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Counter layout shared (by specification, not by code) with the GPU path:
 *   key = (seed & 0xffffffff, seed >> 32)
 *   ctr = (m, c, j, (instance << 20) | (tag << 16) | i)
 * j = 0xffffffff for the START and TEST tags. */
enum { ORA_TAG_START = 0, ORA_TAG_INCR = 1, ORA_TAG_TEST = 2, ORA_TAG_PARAM = 3 };

/* 52-bit uniform in (0,1): n = (a << 20) ^ (b >> 12) (52 bits),
 * u = (2n+1) 2^-53. Exactly representable; min 2^-53, max 1-2^-53. */
double ora_u01(uint32_t a, uint32_t b);

/* d start uniforms of path (i,m) (START tag) and d normals of Euler step j. */
void ora_start_uniforms(uint64_t seed, int instance, int i, uint32_t m, int d, double* u);
void ora_normals(uint64_t seed, int instance, int i, uint32_t m, int j, int d, double* z);
/* d uniforms of test point p at time index i (TEST tag). */
void ora_test_uniforms(uint64_t seed, int instance, int i, uint32_t p, int d, double* u);

/* ---- sampling density nu (Sec. 2.1.2), one 1-D marginal, same for all l. */
enum {
    ORA_NU_LOMAX = 0,    /* (mu/2)(1+|x|)^-(mu+1), "double Lomax" */
    ORA_NU_STUDENT2 = 1, /* 0.5(1+x^2)^-3/2, closed form of Sec. 5 */
    ORA_NU_CAUCHY = 2    /* 1/(pi(1+x^2)) (mu = 1, Sec. 5) */
};
double ora_nu_pdf(int kind, double mu, double x);
double ora_nu_cdf(int kind, double mu, double x);
double ora_nu_icdf(int kind, double mu, double u);

/* ---- driver f and terminal g families */
enum {
    ORA_F_ZERO = 0,
    ORA_F_LINEAR = 1,       /* f = lambda*y                       par = {lambda} */
    ORA_F_CUBIC_MANUF = 2,  /* f = -y^3 + r(t,x)                   par = {a, s_1..s_d} */
    ORA_F_PAPER_MIN = 3     /* f = min(1,[y-k-1-sin(l sum x)e^{l^2 d(t-T)/2}]^2)  par = {kappa, lambda} */
};
enum {
    ORA_GT_COS = 0,         /* g = cos(s.x)                        par = {s_1..s_d} */
    ORA_GT_TRIGPOLY = 1,    /* g = Re sum_k c_k e^{2 pi i k.F(x)}  par = {c re,im interleaved, in Gamma order} */
    ORA_GT_PAPER_SIN = 2    /* g = 1+kappa+sin(lambda sum x)       par = {kappa, lambda} */
};

/* ---- basis (Sec. 2.2): tensor products of 1-D functions of u_l = F_nu(x_l) */
enum {
    ORA_BASIS_FOURIER = 0, /* e^{2 pi i k u}, k in Z (the benchmark workloads) */
    ORA_BASIS_COS = 1      /* C_0 = 1, C_k = sqrt(2) cos(k pi u), k in N (Lemma ortho:dim1) */
};

typedef struct {
    int d, N;
    double T;
    int nu_kind;
    double mu;
    int nG;              /* |Gamma| */
    const int* k;        /* nG*d, canonical order */
    int kmax;            /* max |k_l| over Gamma; <= 0: computed on each use */
    const double* b;     /* d drift, constant */
    const double* sigma; /* d*d row-major, constant */
    int f_kind;
    const double* f_par;
    int g_kind;
    const double* g_par;
    long long M;         /* paths per time index (normalisation 1/M) */
    uint64_t seed;
    int instance;
    double clamp_L;      /* <= 0: no truncation */
    int lattice_n;       /* > 0: start points on the centred lattice (n^d = M) instead of Philox */
    int basis;           /* ORA_BASIS_FOURIER (k in Z^d) or ORA_BASIS_COS (k in N^d, real alpha) */
    double q_damp;       /* damping exponent q of eq. (yqi): the series represents
                          * ybar^q = y / (1 + |x|^2)^{q/2}; 0 = undamped */
} ora_problem;

/* Series y(x) = Re sum_{k in Gamma} alpha_k phi_k(x), phi_k(x) = prod_l e^{2 pi i k_l F(x_l)}
 * (Fourier) or prod_l C_{k_l}(F(x_l)) (cosine); alpha: nG complex, interleaved (re, im). */
double ora_series(const ora_problem* p, const double* alpha, const double* x);
double ora_g(const ora_problem* p, const double* x);
double ora_f(const ora_problem* p, double t, const double* x, double y);

/* Response S_i of path (i,m) under coefficients alpha (N rows of nG complex;
 * row j is ybar_j, j < N). Returns S and writes the start uniforms to u_out (d). */
double ora_response(const ora_problem* p, const double* alpha, int i, long long m,
                    double* u_out, long long* clamp_hits);

/* One Jacobi-Picard iteration on rows i in [i_lo, i_hi) using paths m in
 * [m_lo, m_hi): alpha_out[i] = (1/(m_hi-m_lo)) sum_m S_i^m conj(phi_k(U^m)).
 * alpha_in / alpha_out: N*nG complex interleaved (rows outside [i_lo,i_hi)
 * of alpha_out are left untouched). nthreads <= 0: OpenMP default.
 * Returns 0 on success. */
int ora_picard_iter(const ora_problem* p, const double* alpha_in, double* alpha_out,
                    int i_lo, int i_hi, long long m_lo, long long m_hi,
                    int nthreads, long long* clamp_hits);

/* Backward sweep of Algorithm 1 (i = N-1 .. 0) in place on alpha. */
int ora_backward_sweep(const ora_problem* p, double* alpha, long long m_lo, long long m_hi,
                       int nthreads, long long* clamp_hits);

/* Responses S_i^m for m in [m_lo, m_hi) (debugging / parity of the path kernel). */
int ora_responses(const ora_problem* p, const double* alpha_in, int i,
                  long long m_lo, long long m_hi, double* S_out, int nthreads);

/* Number of OpenMP threads a parallel region would use. */
int ora_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
