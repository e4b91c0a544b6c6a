// qr_device.cuh -- device-side building blocks of the QRMC path (sm_103a).
//
//  * Philox4x32-10 counter generator (Salmon et al., SC'11) and the counter
//    layout of include/qr.h;
//  * 52-bit uniforms kept as integers so that min(u, 1-u) is exact;
//  * the sampling density nu of Sec. 2.1.2 (inverse CDF at the start point,
//    and e^{2 pi i F_nu(x)} at path points without the cancellation of 1-F);
//  * driver / terminal families and the Euler step of Sec. 2.1.1;
//  * bounded mbarrier waits for the bulk (TMA) copies.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "qr_internal.h"

// Checked builds (QR_CHECKED = 1; build.py --checked, libqrmc_checked.so)
// stand in for a memory checker: every kernel index into S, the projection
// partials and the coefficient rows is tested against its buffer; one that
// falls outside sets ST_BOUNDS in the context's status word (the call then
// returns QR_ECUDA) and the access is skipped. In normal builds the test
// folds away.
#ifndef QR_CHECKED
#define QR_CHECKED 0
#endif

namespace qr {

__device__ __forceinline__ bool in_bounds(const QrParams& P, bool ok)
{
#if QR_CHECKED
    if (!ok && P.check) atomicOr(P.check, ST_BOUNDS);
    return ok;
#else
    (void)P;
    (void)ok;
    return true;
#endif
}

template <typename R> struct V2t;
template <> struct V2t<float> { using T = float2; };
template <> struct V2t<double> { using T = double2; };
template <typename R> using V2 = typename V2t<R>::T;

template <typename R> __device__ __forceinline__ V2<R> mk2(R a, R b);
template <> __device__ __forceinline__ float2 mk2<float>(float a, float b) { return make_float2(a, b); }
template <> __device__ __forceinline__ double2 mk2<double>(double a, double b) { return make_double2(a, b); }

// a product the compiler never fuses into an FMA
template <typename R> __device__ __forceinline__ R mul_rn(R a, R b);
template <> __device__ __forceinline__ float mul_rn<float>(float a, float b) { return __fmul_rn(a, b); }
template <> __device__ __forceinline__ double mul_rn<double>(double a, double b) { return __dmul_rn(a, b); }

// complex product with its roundings fixed in the source (one product
// rounded, one fused), so that every kernel inlining it rounds alike
template <typename R>
__device__ __forceinline__ V2<R> cmul(V2<R> a, V2<R> b)
{
    return mk2<R>(fma(a.x, b.x, -mul_rn<R>(a.y, b.y)), fma(a.x, b.y, mul_rn<R>(a.y, b.x)));
}

// ------------------------------------------------------------------ Philox
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t a0 = 0xD2511F53u, a1 = 0xCD9E8D57u;
        uint32_t hi0 = __umulhi(a0, c.x), lo0 = a0 * c.x;
        uint32_t hi1 = __umulhi(a1, c.z), lo1 = a1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ uint32_t ctr_hi(int instance, int tag, int i)
{
    return ((uint32_t)instance << 20) | ((uint32_t)tag << 16) | (uint32_t)i;
}

// 52-bit integer of a uniform u = (2n+1) 2^-53
__device__ __forceinline__ uint64_t u52(uint32_t a, uint32_t b)
{
    return ((uint64_t)a << 20) ^ (uint64_t)(b >> 12);
}
constexpr uint64_t kHalf52 = 1ull << 51;
constexpr uint64_t kTop52 = (1ull << 52) - 1;

__device__ __forceinline__ double u_of(uint64_t n) { return (double)(2 * n + 1) * 0x1p-53; }
// min(u, 1-u) * 2 = (2 min(n, 2^52-1-n) + 1) 2^-52, exact in both types' exponent range
__device__ __forceinline__ uint64_t tail_odd(uint64_t n)
{
    return 2 * (n < kHalf52 ? n : kTop52 - n) + 1;
}

// -------------------------------------------------------------------- nu
// Inverse CDF at the start point, from the integer n of u.
template <typename R>
__device__ __forceinline__ R nu_icdf(const QrParams& P, uint64_t n)
{
    const bool lower = n < kHalf52;
    const uint64_t odd = tail_odd(n);
    if (P.nu_kind == QR_NU_LOMAX) {
        // F^{-1}(u) = sign(u-1/2) ((2w)^{-1/mu} - 1), w = min(u, 1-u)
        R w2 = (R)odd * (R)0x1p-52;
        R x;
        if (P.mu_is3)
            x = (sizeof(R) == 4) ? (R)rcbrtf((float)w2) : (R)rcbrt((double)w2);
        else
            x = (sizeof(R) == 4) ? (R)powf((float)w2, (float)-P.inv_mu) : (R)pow((double)w2, -P.inv_mu);
        x -= (R)1;
        return lower ? -x : x;
    }
    if (P.nu_kind == QR_NU_STUDENT2) {
        // F^{-1}(u) = (u - 1/2)/sqrt(u(1-u))  (closed form of Sec. 5)
        R w = (R)odd * (R)0x1p-53;  // min(u, 1-u)
        R h = (R)0.5 - w;           // |u - 1/2|, exact
        R x = h * ((sizeof(R) == 4) ? (R)rsqrtf((float)(w * ((R)1 - w))) : (R)rsqrt((double)(w * ((R)1 - w))));
        return lower ? -x : x;
    }
    // Cauchy: tan(pi (u - 1/2)) = cot(pi w) in magnitude
    R w = (R)odd * (R)0x1p-53;
    R s, c;
    if (sizeof(R) == 4) {
        float sf, cf;
        sincospif((float)w, &sf, &cf);
        s = sf;
        c = cf;
    } else {
        double sd, cd;
        sincospi((double)w, &sd, &cd);
        s = (R)sd;
        c = (R)cd;
    }
    R x = c / s;
    return lower ? -x : x;
}

// e^{2 pi i F_nu(x)}: with w = F_nu(-|x|) in (0, 1/2], F = w (x < 0) or
// 1 - w (x >= 0), so the phase is e^{+-2 pi i w} with no cancellation.
// For the cosine basis the half angle e^{i pi F} = e^{i pi w} (x < 0) or
// -e^{-i pi w} (x >= 0).
template <typename R>
__device__ __forceinline__ V2<R> nu_phase(const QrParams& P, R x)
{
    R ax = x < (R)0 ? -x : x;
    R w;
    if (P.nu_kind == QR_NU_LOMAX) {
        if (P.mu_is3) {
            R r = (R)1 / ((R)1 + ax);
            w = (R)0.5 * r * r * r;
        } else {
            w = (R)0.5 * ((sizeof(R) == 4) ? (R)powf((float)((R)1 + ax), (float)-P.mu)
                                           : (R)pow((double)((R)1 + ax), -P.mu));
        }
    } else if (P.nu_kind == QR_NU_STUDENT2) {
        R q = (sizeof(R) == 4) ? (R)sqrtf((float)(ax * ax + (R)1)) : (R)sqrt((double)(ax * ax + (R)1));
        w = (R)0.5 / (q * (q + ax));
    } else {
        w = ((sizeof(R) == 4) ? (R)atan2f(1.0f, (float)ax) : (R)atan2(1.0, (double)ax)) * (R)0.3183098861837906715;
    }
    // e^{2 pi i F(x)}, or e^{i pi F(x)} for the cosine basis (half angle);
    // F(x) = w for x < 0 and 1 - w for x >= 0
    const R ang = P.half_angle ? w : (R)2 * w;
    R s, c;
    if (sizeof(R) == 4) {
        float sf, cf;
        sincospif((float)ang, &sf, &cf);
        s = sf;
        c = cf;
    } else {
        double sd, cd;
        sincospi((double)ang, &sd, &cd);
        s = (R)sd;
        c = (R)cd;
    }
    if (P.half_angle) return mk2<R>(x < (R)0 ? c : -c, s);
    return mk2<R>(c, x < (R)0 ? s : -s);
}

// e^{2 pi i u} (or e^{i pi u} when half) for the exact start uniform u = (2n+1) 2^-53
template <typename R>
__device__ __forceinline__ V2<R> u_phase(uint64_t n, bool half)
{
    R w = (R)tail_odd(n) * (R)0x1p-53;  // min(u, 1-u)
    const R ang = half ? w : (R)2 * w;
    R s, c;
    if (sizeof(R) == 4) {
        float sf, cf;
        sincospif((float)ang, &sf, &cf);
        s = sf;
        c = cf;
    } else {
        double sd, cd;
        sincospi((double)ang, &sd, &cd);
        s = (R)sd;
        c = (R)cd;
    }
    if (half) return mk2<R>(n < kHalf52 ? c : -c, s);
    return mk2<R>(c, n < kHalf52 ? s : -s);
}

// ln(u) for u = (2n+1) 2^-53, accurate on both sides of 1/2
template <typename R>
__device__ __forceinline__ R log_u(uint64_t n)
{
    if (n < kHalf52) {
        R u = (R)(2 * n + 1) * (R)0x1p-53;
        return (sizeof(R) == 4) ? (R)logf((float)u) : (R)log((double)u);
    }
    R t = (R)(2 * (kTop52 - n) + 1) * (R)0x1p-53;  // 1 - u, exact
    return (sizeof(R) == 4) ? (R)log1pf(-(float)t) : (R)log1p(-(double)t);
}

// ------------------------------------------------------- sampling per path
// Start uniforms (integers) of path (i, m): call c gives coordinates 2c, 2c+1.
template <int D>
__device__ __forceinline__ void start_ints(const QrParams& P, int i, uint32_t m, uint64_t (&n)[D])
{
    const uint2 key = make_uint2(P.key0, P.key1);
#pragma unroll
    for (int c = 0; 2 * c < D; ++c) {
        uint4 r = philox4x32_10(make_uint4(m, (uint32_t)c, 0xffffffffu, ctr_hi(P.instance, QR_TAG_START, i)), key);
        n[2 * c] = u52(r.x, r.y);
        if (2 * c + 1 < D) n[2 * c + 1] = u52(r.z, r.w);
    }
}

// Brownian increments of step j of path (i, m) (Box-Muller, one pair per call).
template <typename R, int D>
__device__ __forceinline__ void normals(const QrParams& P, int i, uint32_t m, int j, R (&z)[D])
{
    const uint2 key = make_uint2(P.key0, P.key1);
#pragma unroll
    for (int c = 0; 2 * c < D; ++c) {
        uint4 r = philox4x32_10(make_uint4(m, (uint32_t)c, (uint32_t)j, ctr_hi(P.instance, QR_TAG_INCR, i)), key);
        uint64_t na = u52(r.x, r.y), nb = u52(r.z, r.w);
        R rho = (sizeof(R) == 4) ? (R)sqrtf(-2.0f * (float)log_u<R>(na)) : (R)sqrt(-2.0 * (double)log_u<R>(na));
        R ub = (R)(2 * nb + 1) * (R)0x1p-53;
        R s, co;
        if (sizeof(R) == 4) {
            float sf, cf;
            sincospif(2.0f * (float)ub, &sf, &cf);
            s = sf;
            co = cf;
        } else {
            double sd, cd;
            sincospi(2.0 * (double)ub, &sd, &cd);
            s = (R)sd;
            co = (R)cd;
        }
        z[2 * c] = rho * co;
        if (2 * c + 1 < D) z[2 * c + 1] = rho * s;
    }
}

// Start point: exact uniforms (as phases for the basis) and X = F^{-1}(U).
// For the lattice test hook u_l = (digit_l + 1/2)/L.
template <typename R, int D>
__device__ __forceinline__ void start_point(const QrParams& P, int i, long long m, R (&x)[D], V2<R> (&ph)[D],
                                            bool want_phase)
{
    if (P.lattice_n > 0) {
        long long r = m;
#pragma unroll
        for (int l = 0; l < D; ++l) {
            int dig = (int)(r % P.lattice_n);
            r /= P.lattice_n;
            double u = ((double)dig + 0.5) / (double)P.lattice_n;
            double w = u < 0.5 ? u : 1.0 - u;
            double xx;
            if (P.nu_kind == QR_NU_LOMAX) {
                xx = pow(2.0 * w, -P.inv_mu) - 1.0;
            } else if (P.nu_kind == QR_NU_STUDENT2) {
                xx = (0.5 - w) * rsqrt(w * (1.0 - w));
            } else {
                double sd, cd;
                sincospi(w, &sd, &cd);
                xx = cd / sd;
            }
            x[l] = (R)(u < 0.5 ? -xx : xx);
            if (want_phase) {
                double sd, cd;
                sincospi(P.half_angle ? u : 2.0 * u, &sd, &cd);
                ph[l] = mk2<R>((R)cd, (R)sd);
            }
        }
        return;
    }
    uint64_t n[D];
    start_ints<D>(P, i, (uint32_t)m, n);
#pragma unroll
    for (int l = 0; l < D; ++l) {
        x[l] = nu_icdf<R>(P, n[l]);
        if (want_phase) ph[l] = u_phase<R>(n[l], P.half_angle != 0);
    }
}

// Phases e^{2 pi i U_l} of the exact start uniforms of path (i, m)
template <typename R, int D>
__device__ __forceinline__ void start_phases_dev(const QrParams& P, int i, long long m, V2<R> (&ph)[D])
{
    if (P.lattice_n > 0) {
        R x[D];
        start_point<R, D>(P, i, m, x, ph, true);
        return;
    }
    uint64_t n[D];
    start_ints<D>(P, i, (uint32_t)m, n);
#pragma unroll
    for (int l = 0; l < D; ++l) ph[l] = u_phase<R>(n[l], P.half_angle != 0);
}

// Damping of eq. (yqi): the series represents ybar^q = y / w(x),
// w(x) = (1 + |x|^2)^{q/2}. log w with qh = q/2:
template <typename R, int D>
__device__ __forceinline__ R damp_logw(R qh, const R (&x)[D])
{
    R r2 = 0;
#pragma unroll
    for (int l = 0; l < D; ++l) r2 += x[l] * x[l];
    return qh * ((sizeof(R) == 4) ? (R)log1pf((float)r2) : (R)log1p((double)r2));
}

// y w(x) from y and log w, formed in the log domain so that a weight that
// alone would overflow does not (y = 0 stays 0)
template <typename R>
__device__ __forceinline__ R undamp(R y, R lw)
{
    const R a = y < (R)0 ? -y : y;
    if (a == (R)0) return y;
    const R v = (sizeof(R) == 4) ? (R)expf((float)(lw + (R)logf((float)a))) : (R)exp((double)lw + log((double)a));
    return y < (R)0 ? -v : v;
}

// Euler step of Sec. 2.1.1 with constant b and sigma
template <typename R, int D>
__device__ __forceinline__ void euler(const QrParams& P, const R (&x)[D], const R (&z)[D], R (&x1)[D])
{
    const R dt = (R)P.dt, sq = (R)P.sqdt;
#pragma unroll
    for (int l = 0; l < D; ++l) {
        R noise;
        if (P.sig_diag) {
            noise = (R)P.sig[l * D + l] * z[l];
        } else {
            noise = 0;
#pragma unroll
            for (int c = 0; c < D; ++c) noise += (R)P.sig[l * D + c] * z[c];
        }
        x1[l] = x[l] + (R)P.b[l] * dt + noise * sq;
    }
}

template <typename R, int D>
__device__ __forceinline__ R dot_s(const double* s, const R (&x)[D])
{
    R a = 0;
#pragma unroll
    for (int l = 0; l < D; ++l) a += (R)s[l] * x[l];
    return a;
}

template <typename R>
__device__ __forceinline__ R rcos(R a)
{
    return (sizeof(R) == 4) ? (R)cosf((float)a) : (R)cos((double)a);
}
template <typename R>
__device__ __forceinline__ R rsin(R a)
{
    return (sizeof(R) == 4) ? (R)sinf((float)a) : (R)sin((double)a);
}

// driver f(t_j, x, y); fexp[j] holds the time factor of the family
template <typename R, int D>
__device__ __forceinline__ R drv_f(const QrParams& P, int j, const R (&x)[D], R y)
{
    switch (P.f_kind) {
    case QR_F_LINEAR:
        return (R)P.f_lam * y;
    case QR_F_CUBIC_MANUF: {
        R u = (R)P.fexp[j] * rcos<R>(dot_s<R, D>(P.f_s, x));
        return -y * y * y + ((R)P.f_c * u + u * u * u);
    }
    case QR_F_PAPER_MIN: {
        R sx = 0;
#pragma unroll
        for (int l = 0; l < D; ++l) sx += x[l];
        R v = y - (R)P.f_kap - (R)1 - rsin<R>((R)P.f_lam * sx) * (R)P.fexp[j];
        v = v * v;
        return v < (R)1 ? v : (R)1;
    }
    default:
        return (R)0;
    }
}

// terminal g(x) for the closed-form families (the trigonometric polynomial
// is evaluated as a series by the callers)
template <typename R, int D>
__device__ __forceinline__ R term_g(const QrParams& P, const R (&x)[D])
{
    if (P.g_kind == QR_GT_COS) return rcos<R>(dot_s<R, D>(P.g_s, x));
    R sx = 0;
#pragma unroll
    for (int l = 0; l < D; ++l) sx += x[l];
    return (R)1 + (R)P.g_kap + rsin<R>((R)P.g_lam * sx);
}

__device__ __forceinline__ unsigned long long warp_sum_ull(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ------------------------------------------------------ mbarrier / bulk copy
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One elected thread: expect `bytes` and start a bulk global->shared copy.
__device__ __forceinline__ void bulk_load(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Bounded wait for the phase `parity` of an mbarrier. Returns false when
// about 2^31 SM cycles (~1 s) passed without completion.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    const uint32_t a = smem_u32(bar);
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > (1ll << 31)) return false;
    }
}

}  // namespace qr
