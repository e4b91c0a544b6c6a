// qr_tree.cuh -- compile-time chain tree of the |k|_1 <= n and |k|_inf <= n
// half sets and the per-tile body of the path-and-series kernel; used by the
// single-problem kernel (qr_fast.cu) and the multi-instance engine
// (qr_batch.cu).
#pragma once

#include "qr_device.cuh"
#include "qr_fast.h"

// FP32 per-step transcendentals (see nu_phase_fast, rcos_fast and
// normals_fast below): SFU forms on exactly reduced arguments
#ifndef QR_FAST_PHASE
#define QR_FAST_PHASE 1
#endif
#ifndef QR_FAST_BM
#define QR_FAST_BM 0
#endif
#ifndef QR_FAST_FCOS
#define QR_FAST_FCOS 1
#endif
#ifndef QR_FAST_UNI
#define QR_FAST_UNI 1
#endif

namespace qr {

template <int D, int NN, int KIND>
struct TreeShape {
    static constexpr bool ext_ok(int S) { return KIND == QR_G_L1 ? S >= 1 : S < NN; }
    static constexpr int ext_S(int S) { return KIND == QR_G_L1 ? S - 1 : S + 1; }
    static constexpr bool new_ok(int S) { return KIND == QR_G_L1 ? S >= 1 : true; }
    static constexpr int new_S(int S) { return KIND == QR_G_L1 ? S - 1 : 1; }
    static constexpr bool leaf(int L, int S) { return KIND == QR_G_L1 ? S == 0 : (S == NN && L == D - 1); }
    static constexpr int root_S() { return KIND == QR_G_L1 ? NN - 1 : 1; }
    // slots of the subtree of an internal node (L, S), its own slot included
    static constexpr int size(int L, int S)
    {
        int n = 1;
        if (ext_ok(S)) n += leaf(L, ext_S(S)) ? 1 : size(L, ext_S(S));
        if (new_ok(S))
            for (int l2 = L + 1; l2 < D; ++l2) n += leaf(l2, new_S(S)) ? 2 : 2 * size(l2, new_S(S));
        return n;
    }
    static constexpr int total()
    {
        int n = 1;
        for (int l = 0; l < D; ++l) n += leaf(l, root_S()) ? 1 : size(l, root_S());
        return n;
    }
    // slots of a node (D-1, S) of the last dimension: itself and its chain of
    // extensions (a node of the last dimension has no new-dimension children)
    static constexpr int chain_len(int S)
    {
        return 1 + (ext_ok(S) ? (leaf(D - 1, ext_S(S)) ? 1 : chain_len(ext_S(S))) : 0);
    }
    // powers z_{D-1}^m, m = 1..npow, used by the last-dimension pair chains
    static constexpr int npow()
    {
        const int np = KIND == QR_G_L1 ? NN - 1 : NN;
        return np < 1 ? 1 : np;
    }
};

// the phases of one path point as the tree evaluation sees them: z[p][l] =
// e^{2 pi i F(x_l)}, the powers zl[p][m] = z[p][D-1]^{m+1} and, for the pair
// form of dimension l = D-2-v (v < NLV), zk[p][v][m] = z[p][l]^{m+1}
template <typename R, int P, int D, int NPW>
struct TreePh {
    static constexpr int NLV = D - 2 < QR_TREE_PAIR_LEVELS ? (D > 2 ? D - 2 : 0) : QR_TREE_PAIR_LEVELS;
    // dimension L2 (>= 1, a new-dimension child) takes the pair form
    static constexpr bool paired(int L2) { return L2 <= D - 2 && L2 >= D - 1 - NLV; }
    V2<R> z[P][D];
    V2<R> zl[P][NPW];
    V2<R> zk[P][NLV > 0 ? NLV : 1][NPW];
};

template <typename R>
__device__ __forceinline__ void cfma(V2<R>& t, V2<R> c, V2<R> w)
{
    t.x = fma(c.x, w.x, t.x);
    t.x = fma(-c.y, w.y, t.x);
    t.y = fma(c.x, w.y, t.y);
    t.y = fma(c.y, w.x, t.y);
}

// ---- per-step helpers of the tree kernel with the problem constants
// converted once to R (no FP64 instruction per step in the FP32 form)
template <typename R, int D>
struct StepConsts {
    R dt, sqdt, Lc, fc, glam, gkap, flam, fkap, qh;
    R b[D], sig[D * D], fs[D], gs[D];
    bool clamp, sig_diag, damp;
    __device__ __forceinline__ explicit StepConsts(const QrParams& P)
    {
        dt = (R)P.dt;
        sqdt = (R)P.sqdt;
        Lc = (R)P.clamp_L;
        clamp = P.clamp_L > 0.0;
        fc = (R)P.f_c;
        flam = (R)P.f_lam;
        fkap = (R)P.f_kap;
        glam = (R)P.g_lam;
        gkap = (R)P.g_kap;
        sig_diag = P.sig_diag != 0;
        damp = P.q_damp != 0.0;
        qh = (R)(0.5 * P.q_damp);
#pragma unroll
        for (int l = 0; l < D; ++l) {
            b[l] = (R)P.b[l];
            fs[l] = (R)P.f_s[l];
            gs[l] = (R)P.g_s[l];
        }
#pragma unroll
        for (int t = 0; t < D * D; ++t) sig[t] = (R)P.sig[t];
    }
};

// uniform (2n+1) 2^-53, n = (a << 20) ^ (b >> 12), from 32-bit conversions
__device__ __forceinline__ float u01_f32(uint32_t a, uint32_t b)
{
    return fmaf((float)(b >> 12), 0x1p-52f, fmaf((float)a, 0x1p-32f, 0x1p-53f));
}

// The same uniform without integer-to-float conversion instructions (which
// B300 issues to its narrow FP64 pipe): each piece of n below 2^23 becomes
// an exact float by placing it in the mantissa of 2^23 and subtracting 2^23,
// u = (a >> 16) 2^-16 + (a & 0xffff) 2^-32 + (b >> 12) 2^-52 + 2^-53, summed
// by FMA from the smallest piece up (two roundings in all).
__device__ __forceinline__ float u01_bits(uint32_t a, uint32_t b)
{
    const float fh = __uint_as_float(0x4B000000u | (a >> 16)) - 8388608.0f;
    const float fl = __uint_as_float(0x4B000000u | (a & 0xFFFFu)) - 8388608.0f;
    const float fb = __uint_as_float(0x4B000000u | (b >> 12)) - 8388608.0f;
    return fmaf(fh, 0x1p-16f, fmaf(fl, 0x1p-32f, fmaf(fb, 0x1p-52f, 0x1p-53f)));
}

template <typename R, int D>
__device__ __forceinline__ void normals_fast(const QrParams& P, int i, uint32_t m, int j, R (&z)[D])
{
    if constexpr (sizeof(R) == 8) {
        normals<R, D>(P, i, m, j, z);
    } else {
        const uint2 key = make_uint2(P.key0, P.key1);
#pragma unroll
        for (int c = 0; 2 * c < D; ++c) {
            const uint4 r = philox4x32_10(make_uint4(m, (uint32_t)c, (uint32_t)j, ctr_hi(P.instance, QR_TAG_INCR, i)), key);
            // ln(u_a), the same for every lane (no divergent pair of library
            // logarithms): u_a < 1/2 iff the top bit of r.x is clear, and then
            // __logf (at most 3 ulp off [0.5, 2], 2^-21.41 absolute on it);
            // above 1/2, with v = 1 - u_a from the complemented bits,
            // ln(1 - v) = 2 atanh(s), s = -v / (2 - v), |s| < 1/3, by the odd
            // Taylor series of atanh to s^15 (truncation below 2e-9 relative)
#if QR_FAST_UNI
            // t = min(u_a, 1 - u_a) from the integer (complemented words when
            // u_a >= 1/2, exact); ln u_a = ln t or ln(1 - t)
            const bool upper = (r.x & 0x80000000u) != 0;
            const float v = u01_bits(upper ? ~r.x : r.x, upper ? ~r.y : r.y);
#else
            const float v = u01_f32(~r.x, ~r.y);
#endif
            const float s = __fdividef(-v, 2.0f - v), s2 = s * s;
            float t = 1.0f / 15.0f;
            t = fmaf(t, s2, 1.0f / 13.0f);
            t = fmaf(t, s2, 1.0f / 11.0f);
            t = fmaf(t, s2, 1.0f / 9.0f);
            t = fmaf(t, s2, 1.0f / 7.0f);
            t = fmaf(t, s2, 1.0f / 5.0f);
            t = fmaf(t, s2, 1.0f / 3.0f);
            t = fmaf(t, s2, 1.0f);
#if QR_FAST_UNI
            const float la = upper ? 2.0f * s * t : __logf(v);
            const float rr = -2.0f * la;  // >= 2^-52 > 0
            const float rho = rr * rsqrtf(rr);
            const float ub = u01_bits(r.z, r.w);
#else
            const float la = (r.x & 0x80000000u) ? 2.0f * s * t : __logf(u01_f32(r.x, r.y));
            const float rho = sqrtf(-2.0f * la);
            const float ub = u01_f32(r.z, r.w);
#endif
            float sn, cs;
#if QR_FAST_BM
            // (cos, sin)(2 pi u_b) = -(cos, sin)(2 pi (u_b - 1/2)), argument in [-pi, pi]
            __sincosf(6.28318530717958648f * (ub - 0.5f), &sn, &cs);
            sn = -sn;
            cs = -cs;
#else
            sincospif(2.0f * ub, &sn, &cs);
#endif
            z[2 * c] = rho * cs;
            if (2 * c + 1 < D) z[2 * c + 1] = rho * sn;
        }
    }
}

// ---- FP32 per-step transcendentals of the tree path kernels
// The phases e^{2 pi i F(x)} of the series and the cosine of the driver are
// evaluated with the SFU's sine/cosine (__sincosf, __cosf: absolute error at
// most 2^-21.41 on [-pi, pi]) on arguments reduced to that range exactly:
//  * phase: with w = F(-|x|) = (1/2)(1+|x|)^-3 in (0, 1/2] (double Lomax,
//    mu = 3), the angle 2 pi w lies in (0, pi] with no reduction, and
//    e^{2 pi i F(x)} = e^{-+2 pi i w} for x >= 0 / x < 0; the reciprocal is
//    the SFU's (__fdividef, 2 ulp);
//  * cosine of an argument a: Cody-Waite reduction r = a - 2 pi rint(a/2pi)
//    with 2 pi split into a float and its float remainder, each product
//    exact inside an FMA, so |r| <= pi + 1e-6 for |a| < 2^20; larger |a|
//    (far tails of the start law) take the library cosf.

template <typename R>
__device__ __forceinline__ V2<R> nu_phase_fast(const QrParams& P, R x)
{
#if QR_FAST_PHASE
    if constexpr (sizeof(R) == 4) {
        if (P.nu_kind == QR_NU_LOMAX && P.mu_is3 && !P.half_angle) {
            const float ax = fabsf(x);
            const float r = __fdividef(1.0f, 1.0f + ax);
            const float w = 0.5f * r * r * r;
            float sn, cs;
            __sincosf(6.28318530717958648f * w, &sn, &cs);
            return make_float2(cs, x < 0.0f ? sn : -sn);
        }
    }
#endif
    return nu_phase<R>(P, x);
}

template <typename R>
__device__ __forceinline__ R rcos_fast(R a)
{
#if QR_FAST_FCOS
    if constexpr (sizeof(R) == 4) {
        if (fabsf(a) < 1048576.0f) {
            // nearest integer to a/(2 pi) (|.| < 2^18): adding and removing
            // 1.5 2^23 rounds to an integer in the FMA pipe
            const float k = fmaf(a, 0.159154943091895336f, 12582912.0f) - 12582912.0f;
            float r = fmaf(-k, 6.28318548202514648f, a);  // float(2 pi)
            r = fmaf(-k, -1.74845553146951715e-7f, r);    // 2 pi - float(2 pi)
            return __cosf(r);
        }
        return cosf(a);
    }
#endif
    return rcos<R>(a);
}

template <typename R, int D>
__device__ __forceinline__ void euler_fast(const StepConsts<R, D>& K, const R (&x)[D], const R (&z)[D], R (&x1)[D])
{
#pragma unroll
    for (int l = 0; l < D; ++l) {
        R noise;
        if (K.sig_diag) {
            noise = K.sig[l * D + l] * z[l];
        } else {
            noise = 0;
#pragma unroll
            for (int c = 0; c < D; ++c) noise += K.sig[l * D + c] * z[c];
        }
        x1[l] = x[l] + K.b[l] * K.dt + noise * K.sqdt;
    }
}

template <typename R, int D>
__device__ __forceinline__ R drv_f_fast(const QrParams& P, const StepConsts<R, D>& K, R fexp_j, const R (&x)[D], R y)
{
    switch (P.f_kind) {
    case QR_F_LINEAR:
        return K.flam * y;
    case QR_F_CUBIC_MANUF: {
        R sx = 0;
#pragma unroll
        for (int l = 0; l < D; ++l) sx += K.fs[l] * x[l];
        const R u = fexp_j * rcos_fast<R>(sx);
        return -y * y * y + (K.fc * u + u * u * u);
    }
    case QR_F_PAPER_MIN: {
        R sx = 0;
#pragma unroll
        for (int l = 0; l < D; ++l) sx += x[l];
        R v = y - K.fkap - (R)1 - rsin<R>(K.flam * sx) * fexp_j;
        v = v * v;
        return v < (R)1 ? v : (R)1;
    }
    default:
        return (R)0;
    }
}

template <typename R, int D>
__device__ __forceinline__ R term_g_fast(const QrParams& P, const StepConsts<R, D>& K, const R (&x)[D])
{
    R sx = 0;
    if (P.g_kind == QR_GT_COS) {
#pragma unroll
        for (int l = 0; l < D; ++l) sx += K.gs[l] * x[l];
        return rcos_fast<R>(sx);
    }
#pragma unroll
    for (int l = 0; l < D; ++l) sx += x[l];
    return (R)1 + K.gkap + rsin<R>(K.glam * sx);
}

// +-1 leaf pairs of the FP32 form as two packed two-lane FMA per path
// (__ffma2_rn: the same roundings as four scalar FMA, half the issue slots)
#ifndef QR_TREE_PAIR2
#define QR_TREE_PAIR2 1
#endif

// subtrees of at most this many slots have both signs unrolled (d = 6
// workload with the pair forms, where only the first dimensions' subtrees
// take this branch: 16: 490-492 ms against 499 for 4, 492 for 8 or 32, 496
// for 2, 574 with every subtree unrolled)
#ifndef QR_TREE_UNROLL
#define QR_TREE_UNROLL 16
#endif
constexpr int kUnrollSlots = QR_TREE_UNROLL;

template <typename R, int D, int NN, int KIND, int P, int L, int S>
struct Node;

// t += w v (complex), 4 FMA
template <typename R>
__device__ __forceinline__ void cmad(V2<R>& t, V2<R> w, V2<R> v)
{
    t.x = fma(w.x, v.x, t.x);
    t.x = fma(-w.y, v.y, t.x);
    t.y = fma(w.x, v.y, t.y);
    t.y = fma(w.y, v.x, t.y);
}

// Bottom-up (Horner) evaluation: the value of the subtree of node c in its
// own frame is V_c = coef_c + sum_children w_ch V_ch, and the series is
// Re V_root. Every tree edge costs one complex FMA (4 FMA); a +-1 leaf pair
// costs 4 FMA for both leaves; no prefix products are formed.

// T += c+ w + c- conj(w) for a pair of coefficients at the mirrored
// positions k +- (a step of phase w), pre-combined as the slots (A, C), (B, E):
// T.x += A w.x + B w.y,  T.y += C w.y + E w.x, i.e.
// T += (A, C) * (w.x, w.y) + (B, E) * (w.y, w.x) lane-wise; 4 FMA for two
// coefficients, the sum being real-linear in (Re w, Im w)
template <typename R>
__device__ __forceinline__ void pair_acc(V2<R>& T, V2<R> ac, V2<R> be, V2<R> w)
{
#if QR_TREE_PAIR2
    if constexpr (sizeof(R) == 4) {
        T = __ffma2_rn(ac, w, T);
        T = __ffma2_rn(be, make_float2(w.y, w.x), T);
        return;
    }
#endif
    T.x = fma(ac.x, w.x, T.x);
    T.x = fma(be.x, w.y, T.x);
    T.y = fma(ac.y, w.y, T.y);
    T.y = fma(be.y, w.x, T.y);
}

// T += Re(w) A + Im(w) B, 4 FMA (two packed in the FP32 form)
template <typename R>
__device__ __forceinline__ void rs_acc(V2<R>& T, V2<R> A, V2<R> B, V2<R> w)
{
#if QR_TREE_PAIR2
    if constexpr (sizeof(R) == 4) {
        T = __ffma2_rn(A, make_float2(w.x, w.x), T);
        T = __ffma2_rn(B, make_float2(w.y, w.y), T);
        return;
    }
#endif
    T.x = fma(A.x, w.x, T.x);
    T.y = fma(A.y, w.x, T.y);
    T.x = fma(B.x, w.y, T.x);
    T.y = fma(B.y, w.y, T.y);
}

template <typename R, int D, int NN, int KIND, int P, int L2, int S>
struct NewDims;

// The + and - chains k +- m e_L of a paired dimension L below a node
// (position MM = m - 1 of the chain, node state S2). With U+-_m the subtree
// values at k +- m e_L without their extensions (both in the phases of the
// later dimensions) the chains contribute
//   sum_m (w^m U+_m + conj(w)^m U-_m) = sum_m (Re(w^m) A_m + Im(w^m) B_m),
// A_m = U+_m + U-_m, B_m = i (U+_m - U-_m), both evaluated as subtrees of
// the same shape from pre-combined coefficients; each mirrored pair of
// nodes then costs 4 FMA against the powers w^m instead of two Horner edges.
template <typename R, int D, int NN, int KIND, int P, int L, int S2, int MM>
struct PairChain {
    using Sh = TreeShape<D, NN, KIND>;
    using Ph = TreePh<R, P, D, Sh::npow()>;
    static __device__ __forceinline__ void run(const V2<R>* __restrict__ c, int& off, V2<R> (&T)[P], const Ph& z)
    {
        static_assert(MM < Sh::npow(), "power table too short");
        V2<R> A[P], B[P];
        const V2<R> ca = c[off], cb = c[off + 1];
        off += 2;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            A[p] = ca;
            B[p] = cb;
        }
        if constexpr (!Sh::leaf(L, S2) && Sh::new_ok(S2)) {
            NewDims<R, D, NN, KIND, P, L + 1, S2>::run(c, off, A, z);
            NewDims<R, D, NN, KIND, P, L + 1, S2>::run(c, off, B, z);
        }
#pragma unroll
        for (int p = 0; p < P; ++p) rs_acc<R>(T[p], A[p], B[p], z.zk[p][D - 2 - L][MM]);
        if constexpr (!Sh::leaf(L, S2) && Sh::ext_ok(S2))
            PairChain<R, D, NN, KIND, P, L, Sh::ext_S(S2), MM + 1>::run(c, off, T, z);
    }
};

// children in the new dimensions L2 .. D-1 of a node in state S
template <typename R, int D, int NN, int KIND, int P, int L2, int S>
struct NewDims {
    using Sh = TreeShape<D, NN, KIND>;
    using Ph = TreePh<R, P, D, Sh::npow()>;
    static __device__ __forceinline__ void run(const V2<R>* __restrict__ c, int& off, V2<R> (&T)[P], const Ph& z)
    {
        if constexpr (L2 < D) {
            constexpr int S2 = Sh::new_S(S);
            if constexpr (Sh::leaf(L2, S2)) {
                const V2<R> ac = c[off], be = c[off + 1];
#pragma unroll
                for (int p = 0; p < P; ++p) pair_acc<R>(T[p], ac, be, z.z[p][L2]);
                off += 2;
            } else if constexpr (L2 == D - 1) {
                // the + and - chains k +- m e_{D-1}, m = 1..len, of the last
                // dimension: their contribution in this node's frame,
                // sum_m (c+_m z^m + c-_m conj(z)^m), is real-linear in the
                // powers z^m (computed once per point), so each mirrored pair
                // costs 4 FMA instead of two Horner edges (8 FMA)
                constexpr int len = Sh::chain_len(S2);
                static_assert(len <= Sh::npow(), "power table too short");
#pragma unroll
                for (int mm = 0; mm < len; ++mm) {
                    const V2<R> ac = c[off + 2 * mm], be = c[off + 2 * mm + 1];
#pragma unroll
                    for (int p = 0; p < P; ++p) pair_acc<R>(T[p], ac, be, z.zl[p][mm]);
                }
                off += 2 * len;
            } else if constexpr (Ph::paired(L2)) {
                PairChain<R, D, NN, KIND, P, L2, S2, 0>::run(c, off, T, z);
            } else {
                constexpr int sz = Sh::size(L2, S2);
                const V2<R>* cs = c + off;
                if constexpr (sz <= kUnrollSlots) {
                    // small subtrees: both signs unrolled (no loop control)
                    V2<R> w[P], v[P];
#pragma unroll
                    for (int p = 0; p < P; ++p) w[p] = z.z[p][L2];
                    Node<R, D, NN, KIND, P, L2, S2>::value(cs, w, z, v);
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        cmad<R>(T[p], w[p], v[p]);
                        w[p].y = -w[p].y;
                    }
                    Node<R, D, NN, KIND, P, L2, S2>::value(cs + sz, w, z, v);
#pragma unroll
                    for (int p = 0; p < P; ++p) cmad<R>(T[p], w[p], v[p]);
                } else {
#pragma unroll 1
                    for (int s = 0; s < 2; ++s) {
                        V2<R> w[P], v[P];
#pragma unroll
                        for (int p = 0; p < P; ++p) {
                            w[p] = z.z[p][L2];
                            if (s) w[p].y = -w[p].y;
                        }
                        Node<R, D, NN, KIND, P, L2, S2>::value(cs + s * sz, w, z, v);
#pragma unroll
                        for (int p = 0; p < P; ++p) cmad<R>(T[p], w[p], v[p]);
                    }
                }
                off += 2 * sz;
            }
            NewDims<R, D, NN, KIND, P, L2 + 1, S>::run(c, off, T, z);
        }
    }
};

// an internal node (L, S) reached through the phase wl: its slot, then the
// extension child (same dimension, same phase), then the new dimensions
template <typename R, int D, int NN, int KIND, int P, int L, int S>
struct Node {
    using Sh = TreeShape<D, NN, KIND>;
    using Ph = TreePh<R, P, D, Sh::npow()>;
    static __device__ __forceinline__ void value(const V2<R>* __restrict__ c, const V2<R> (&wl)[P], const Ph& z,
                                                 V2<R> (&T)[P])
    {
        const V2<R> c0 = c[0];
#pragma unroll
        for (int p = 0; p < P; ++p) T[p] = c0;
        int off = 1;
        if constexpr (Sh::ext_ok(S)) {
            constexpr int S2 = Sh::ext_S(S);
            if constexpr (Sh::leaf(L, S2)) {
                const V2<R> ce = c[off];
#pragma unroll
                for (int p = 0; p < P; ++p) cfma<R>(T[p], ce, wl[p]);
                off += 1;
            } else {
                V2<R> v[P];
                Node<R, D, NN, KIND, P, L, S2>::value(c + off, wl, z, v);
#pragma unroll
                for (int p = 0; p < P; ++p) cmad<R>(T[p], wl[p], v[p]);
                off += Sh::size(L, S2);
            }
        }
        if constexpr (Sh::new_ok(S)) NewDims<R, D, NN, KIND, P, L + 1, S>::run(c, off, T, z);
    }
};

// root children (first nonzero coordinate, sign +)
template <typename R, int D, int NN, int KIND, int P, int L>
struct RootKids {
    using Sh = TreeShape<D, NN, KIND>;
    using Ph = TreePh<R, P, D, Sh::npow()>;
    static __device__ __forceinline__ void run(const V2<R>* __restrict__ c, int& off, V2<R> (&T)[P], const Ph& z)
    {
        if constexpr (L < D) {
            constexpr int S0 = Sh::root_S();
            if constexpr (Sh::leaf(L, S0)) {
                const V2<R> ce = c[off];
#pragma unroll
                for (int p = 0; p < P; ++p) cfma<R>(T[p], ce, z.z[p][L]);
                off += 1;
            } else {
                V2<R> w[P], v[P];
#pragma unroll
                for (int p = 0; p < P; ++p) w[p] = z.z[p][L];
                Node<R, D, NN, KIND, P, L, S0>::value(c + off, w, z, v);
#pragma unroll
                for (int p = 0; p < P; ++p) cmad<R>(T[p], w[p], v[p]);
                off += Sh::size(L, S0);
            }
            RootKids<R, D, NN, KIND, P, L + 1>::run(c, off, T, z);
        }
    }
};

template <typename R, int D, int NN, int KIND, int P>
__device__ __forceinline__ void tree_series(const V2<R>* __restrict__ c, const V2<R> (&z)[P][D], R (&y)[P])
{
    using Sh = TreeShape<D, NN, KIND>;
    TreePh<R, P, D, Sh::npow()> ph;
#pragma unroll
    for (int p = 0; p < P; ++p) {
#pragma unroll
        for (int l = 0; l < D; ++l) ph.z[p][l] = z[p][l];
        ph.zl[p][0] = z[p][D - 1];
#pragma unroll
        for (int m = 1; m < Sh::npow(); ++m) ph.zl[p][m] = cmul<R>(ph.zl[p][m - 1], z[p][D - 1]);
#pragma unroll
        for (int v = 0; v < decltype(ph)::NLV; ++v) {
            const V2<R> w = z[p][D - 2 - v];
            ph.zk[p][v][0] = w;
#pragma unroll
            for (int m = 1; m < Sh::npow(); ++m) ph.zk[p][v][m] = cmul<R>(ph.zk[p][v][m - 1], w);
        }
    }
    V2<R> T[P];
    const V2<R> c0 = c[0];
#pragma unroll
    for (int p = 0; p < P; ++p) T[p] = c0;
    int off = 1;
    RootKids<R, D, NN, KIND, P, 0>::run(c, off, T, ph);
#pragma unroll
    for (int p = 0; p < P; ++p) y[p] = T[p].x;
}


// One work item of the path-and-series kernel: the tile of BS*P paths
// starting at path m0 (this thread: m0 + p*BS) of time index i. Coefficient
// rows i+1.. are staged into the two buffers abuf (row i+1 into abuf[0]);
// phase[] carries the mbarrier parities across the items a CTA processes.
// Returns false when a bounded wait ran out (the status word is set).
template <typename R, int D, int NN, int KIND, int P, int BS>
__device__ __forceinline__ bool path_item(const QrParams& Pm, const V2<R>* __restrict__ tree, long long row_stride,
                                          R* __restrict__ S, int i, int i_lo, long long m0, V2<R>* const (&abuf)[2],
                                          uint64_t* bars, uint32_t (&phase)[2],
                                          unsigned long long* __restrict__ counters, unsigned* __restrict__ status)
{
    const int tid = threadIdx.x, N = Pm.N;
    const bool trig = Pm.g_kind == QR_GT_TRIGPOLY;
    const uint32_t rowbytes = (uint32_t)(row_stride * sizeof(V2<R>));
    // the two buffers' pointers, mbarrier parities and in-flight flags, kept
    // in registers (selected by the step parity instead of indexed arrays,
    // which would live in local memory)
    V2<R>* const buf0 = abuf[0];
    V2<R>* const buf1 = abuf[1];
    uint32_t par0 = phase[0], par1 = phase[1];
    bool infl0 = false, infl1 = false;
    if (i + 1 < N || (i + 1 == N && trig)) {
        if (tid == 0) {
            fence_proxy_async_smem();
            bulk_load(buf0, tree + (size_t)(i + 1) * row_stride, rowbytes, &bars[0]);
        }
        infl0 = true;
    }

    const StepConsts<R, D> K(Pm);
    R x[P][D], sum[P], comp[P], gN[P], lw0[P];
    unsigned long long hits = 0;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        V2<R> unused[D];
        start_point<R, D>(Pm, i, m0 + p * BS, x[p], unused, false);
        sum[p] = comp[p] = gN[p] = 0;
        lw0[p] = K.damp ? damp_logw<R, D>(K.qh, x[p]) : (R)0;  // log w(X_i^i), eq. (yqi)
    }
    const R dt = K.dt;

    for (int j = i; j < N; ++j) {
        const int buf = (j - i) & 1, row = j + 1;
        V2<R>* const cur = buf ? buf1 : buf0;
        V2<R>* const nxt = buf ? buf0 : buf1;
        const bool use_series = row < N || trig;
        const int nrow = row + 1;
        R fexp_j;
        if constexpr (sizeof(R) == 4)
            fexp_j = Pm.fexp32[j];
        else
            fexp_j = Pm.fexp[j];
        if (nrow < N || (nrow == N && trig)) {
            if (tid == 0) {
                fence_proxy_async_smem();
                bulk_load(nxt, tree + (size_t)nrow * row_stride, rowbytes, &bars[buf ^ 1]);
            }
            if (buf) infl0 = true;
            else infl1 = true;
        }
        R x1[P][D], y[P];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            R z[D];
            normals_fast<R, D>(Pm, i, (uint32_t)(m0 + p * BS), j, z);
            euler_fast<R, D>(K, x[p], z, x1[p]);
        }
        if (use_series) {
            const bool ok = mbar_wait(&bars[buf], buf ? par1 : par0);
            if (buf) {
                par1 ^= 1u;
                infl1 = false;
            } else {
                par0 ^= 1u;
                infl0 = false;
            }
            if (!__syncthreads_and(ok)) {
                if (tid == 0) {
                    atomicOr(status, ST_TIMEOUT);
                    if (buf ? infl0 : infl1) (void)mbar_wait(&bars[buf ^ 1], buf ? par0 : par1);
                }
                __syncthreads();
                phase[0] = par0;
                phase[1] = par1;
                return false;
            }
            V2<R> zz[P][D];
#pragma unroll
            for (int p = 0; p < P; ++p)
#pragma unroll
                for (int l = 0; l < D; ++l) zz[p][l] = nu_phase_fast<R>(Pm, x1[p][l]);
            tree_series<R, D, NN, KIND, P>(cur, zz, y);
            if (K.damp && row < N) {
#pragma unroll
                for (int p = 0; p < P; ++p) y[p] = undamp<R>(y[p], damp_logw<R, D>(K.qh, x1[p]));
            }
            if (row < N && K.clamp) {
                const R Lc = K.Lc;
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    if (y[p] > Lc) {
                        y[p] = Lc;
                        if (m0 + p * BS < Pm.M) ++hits;
                    } else if (y[p] < -Lc) {
                        y[p] = -Lc;
                        if (m0 + p * BS < Pm.M) ++hits;
                    }
                }
            }
        } else {
#pragma unroll
            for (int p = 0; p < P; ++p) y[p] = term_g_fast<R, D>(Pm, K, x1[p]);
        }
#pragma unroll
        for (int p = 0; p < P; ++p) {
            if (row == N) gN[p] = y[p];
            const R term = drv_f_fast<R, D>(Pm, K, fexp_j, x[p], y[p]) * dt;
            const R yk = term - comp[p];
            const R tk = sum[p] + yk;
            comp[p] = (tk - sum[p]) - yk;
            sum[p] = tk;
#pragma unroll
            for (int l = 0; l < D; ++l) x[p][l] = x1[p][l];
        }
        __syncthreads();
    }
    unsigned long long bad = 0;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const long long m = m0 + p * BS;
        if (m < Pm.M) {
            const R Sv = K.damp ? (gN[p] + sum[p]) * (R)exp((double)-lw0[p]) : gN[p] + sum[p];
            if (in_bounds(Pm, i - i_lo >= 0 && i - i_lo < Pm.N))
                S[(size_t)(i - i_lo) * (size_t)Pm.M + (size_t)m] = Sv;
            if (!isfinite(Sv)) ++bad;
        }
    }
    hits = warp_sum_ull(hits);
    bad = warp_sum_ull(bad);
    if ((tid & 31) == 0) {
        if (hits) atomicAdd(&counters[CNT_CLAMP], hits);
        if (bad) atomicAdd(&counters[CNT_NONFINITE], bad);
    }
    phase[0] = par0;
    phase[1] = par1;
    return true;
}

// ------------------------------------------------------ path-and-series kernel
// resident CTAs per SM the register allocation is held to. FP32: 4 (128
// registers, 16 warps per SM; the d = 6 kernel spills 28 bytes and runs
// 427 ms against 437.5 at 3 CTAs with 158 registers, 604 at 2 CTAs with
// three paths per thread); a file whose classes need more registers sets 3
// before including this header. FP64 (one path per thread): 3. Left free,
// ptxas takes 255 registers (8 warps per SM).
#ifndef QR_TREE_MINB
#define QR_TREE_MINB 4
#endif
#ifndef QR_TREE_MINB64
#define QR_TREE_MINB64 3
#endif
template <typename R, int D, int NN, int KIND, int P, int BS>
__global__ void __launch_bounds__(BS, sizeof(R) == 4 ? QR_TREE_MINB : QR_TREE_MINB64) k_paths_tree(const __grid_constant__ QrParams P_, const V2<R>* __restrict__ tree,
                                                   long long row_stride, R* __restrict__ S, int i_lo,
                                                   int tiles_per_i, unsigned long long* __restrict__ counters,
                                                   unsigned* __restrict__ status)
{
    const QrParams& Pm = P_;
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t rowbytes = (uint32_t)(row_stride * sizeof(V2<R>));
    V2<R>* const abuf[2] = {reinterpret_cast<V2<R>*>(smem), reinterpret_cast<V2<R>*>(smem + rowbytes)};
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * (size_t)rowbytes);
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase[2] = {0u, 0u};
    const int i = i_lo + (int)(blockIdx.x / tiles_per_i);
    const long long m0 = shard_m_lo(Pm) + (long long)(blockIdx.x % tiles_per_i) * (BS * P) + threadIdx.x;
    (void)path_item<R, D, NN, KIND, P, BS>(Pm, tree, row_stride, S, i, i_lo, m0, abuf, bars, phase, counters, status);
}

template <int D, int NN, int KIND>
int tree_slots_t()
{
    return TreeShape<D, NN, KIND>::total();
}

template <typename R, int D, int NN, int KIND>
inline cudaError_t paths_tree_t(const QrParams& P, const void* tree, long long row_stride, void* S, int i_lo,
                                int i_hi, unsigned long long* counters, unsigned* status, cudaStream_t st)
{
#ifndef QR_TREE_P32
#define QR_TREE_P32 2
#endif
    constexpr int PP = sizeof(R) == 4 ? QR_TREE_P32 : 1;  // paths per thread
    constexpr int BS = 128;
    const size_t sm = 2 * (size_t)row_stride * sizeof(V2<R>) + 16;
    if (sm > 227 * 1024) return cudaErrorInvalidConfiguration;
    auto kern = k_paths_tree<R, D, NN, KIND, PP, BS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    // the paths of the context's chunk range (a multiple of the tile: chunks
    // are multiples of 256 paths in FP32 and 128 in FP64)
    const long long span = shard_m_hi(P) - shard_m_lo(P);
    const int tiles = (int)((span + BS * PP - 1) / (BS * PP));
    const long long blocks = (long long)tiles * (i_hi - i_lo);
    if (blocks <= 0) return cudaSuccess;
    kern<<<(unsigned)blocks, BS, sm, st>>>(P, static_cast<const V2<R>*>(tree), row_stride, static_cast<R*>(S), i_lo,
                                           tiles, counters, status);
    return cudaGetLastError();
}


}  // namespace qr
