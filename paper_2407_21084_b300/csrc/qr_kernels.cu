// qr_kernels.cu -- the QRMC Picard iteration on sm_103a.
//
// One iteration is three kernels on one stream:
//   k_paths    path-and-series kernel: for every time index i and path m,
//              draw X_i^i ~ nu, run the Euler path (Sec. 2.1.1) and evaluate
//              the previous iterate ybar_{j+1} at every path point as the
//              series Re sum_k alpha_{j+1,k} phi_k (Algorithm 1, eq. yqi:bar:M)
//              to form the response S_i (eq. Sqi:bar:M). alpha_{j+1} is staged
//              in shared memory by bulk (TMA) copies, double buffered.
//   k_project  projection of the responses on the basis (eq. Aqi:bar:M):
//              per CTA, sum_m S_i^m conj(phi_k(U^m)) over a fixed chunk of
//              paths (warp shuffle tree, then a fixed warp order), written as
//              FP64 partials. U is regenerated from the counter-based
//              generator instead of being stored (Sec. 4 notes the same
//              trade for its multi-GPU variant).
//   k_reduce   deterministic cross-block sum of the partials in FP64, in a
//              fixed chunk order, divided by M; writes alpha (FP64 master),
//              the packed working copy for the next iteration and the
//              iteration residual.
// The basis is evaluated from per-dimension power tables z_l^a, a = 0..K,
// built by complex recurrence from z_l = e^{2 pi i F_nu(x_l)}, with the
// tensor products formed in registers along the canonical order of the half
// set Gamma_+ (entries sharing a prefix of k reuse its partial product).
#include <cstdio>

#include "qr_device.cuh"
#include "qr_reduce.cuh"

namespace qr {

__host__ __device__ __forceinline__ size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

// ----------------------------------------------------------- basis helpers
template <typename R, int D>
__device__ __forceinline__ void fill_powers(V2<R>* pw, int K1, int stride, const V2<R> (&z)[D])
{
#pragma unroll
    for (int l = 0; l < D; ++l) {
        V2<R> p = z[l];
        pw[(l * K1) * stride] = mk2<R>((R)1, (R)0);
        for (int a = 1; a < K1; ++a) {
            pw[(l * K1 + a) * stride] = p;
            p = cmul<R>(p, z[l]);
        }
    }
}

// Advance the prefix products b[] to table entry e (dimensions >= f change).
template <typename R, int D>
__device__ __forceinline__ void basis_step(V2<R> (&b)[D], const GEntry& g, int f, const V2<R>* pw, int K1,
                                           int stride)
{
#pragma unroll
    for (int l = 0; l < D; ++l) {
        if (l >= f) {
            const int v = g.template kv<D>(l);
            V2<R> prev = (l == 0) ? mk2<R>((R)1, (R)0) : b[l - 1];
            if (v == 0) {
                b[l] = prev;
            } else {
                const int a = v < 0 ? -v : v;
                V2<R> p = pw[(l * K1 + a) * stride];
                if (v < 0) p.y = -p.y;
                b[l] = (l == 0) ? p : cmul<R>(prev, p);
            }
        }
    }
}

// ybar(x) = Re sum_e coef[e] b_e(x); coef[0] = alpha_0, coef[e>0] = 2 alpha_k.
template <typename R, int D>
__device__ __forceinline__ R series(const V2<R>* __restrict__ coef, const GEntry* __restrict__ tab,
                                    const uint8_t* __restrict__ first, int nGp, const V2<R>* pw, int K1,
                                    int stride)
{
    V2<R> b[D];
    R acc0 = 0, acc1 = 0;
    int e = 0;
    for (; e + 1 < nGp; e += 2) {
        basis_step<R, D>(b, tab[e], first[e], pw, K1, stride);
        const V2<R> c0 = coef[e];
        acc0 += c0.x * b[D - 1].x - c0.y * b[D - 1].y;
        basis_step<R, D>(b, tab[e + 1], first[e + 1], pw, K1, stride);
        const V2<R> c1 = coef[e + 1];
        acc1 += c1.x * b[D - 1].x - c1.y * b[D - 1].y;
    }
    if (e < nGp) {
        basis_step<R, D>(b, tab[e], first[e], pw, K1, stride);
        const V2<R> c0 = coef[e];
        acc0 += c0.x * b[D - 1].x - c0.y * b[D - 1].y;
    }
    return acc0 + acc1;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ------------------------------------------------------ path-and-series kernel
// TG: the table of multi-indices is read from global memory (warp-uniform,
// L1-cached loads) instead of being copied to shared memory, for index sets
// whose table would not leave room for the power tables and coefficient rows
template <typename R, int D, int BS, bool TG>
__global__ void __launch_bounds__(BS) k_paths(const __grid_constant__ QrParams P, const GEntry* __restrict__ gtab,
                                              const uint8_t* __restrict__ gfirst,
                                              const V2<R>* __restrict__ packed, long long row_stride,
                                              R* __restrict__ S, int i_lo, int tiles_per_i,
                                              unsigned long long* __restrict__ counters,
                                              unsigned* __restrict__ status)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int nGp = P.nGp, K1 = P.K1, N = P.N;
    const uint32_t rowbytes = (uint32_t)(row_stride * sizeof(V2<R>));
    size_t off = 0;
    GEntry* stab = reinterpret_cast<GEntry*>(smem + off);
    if (!TG) off += align16((size_t)nGp * sizeof(GEntry));
    uint8_t* sfirst = smem + off;
    if (!TG) off += align16((size_t)nGp);
    const GEntry* tab = TG ? gtab : stab;
    const uint8_t* first = TG ? gfirst : sfirst;
    V2<R>* abuf[2];
    abuf[0] = reinterpret_cast<V2<R>*>(smem + off);
    off += rowbytes;
    abuf[1] = reinterpret_cast<V2<R>*>(smem + off);
    off += rowbytes;
    V2<R>* pw = reinterpret_cast<V2<R>*>(smem + off);
    off += (size_t)D * K1 * BS * sizeof(V2<R>);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + off);

    const int tid = threadIdx.x;
    const int i = i_lo + (int)(blockIdx.x / tiles_per_i);
    const long long m = shard_m_lo(P) + (long long)(blockIdx.x % tiles_per_i) * BS + tid;
    const bool active = m < P.M;
    const bool trig = P.g_kind == QR_GT_TRIGPOLY;

    if (!TG)
        for (int e = tid; e < nGp; e += BS) {
            stab[e] = gtab[e];
            sfirst[e] = gfirst[e];
        }
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // rows i+1 .. N are read as series (row N only for a polynomial g)
    // buffer state in registers, selected by the step parity (indexed arrays
    // would live in local memory)
    bool infl0 = false, infl1 = false;
    uint32_t par0 = 0u, par1 = 0u;
    if (i + 1 < N || (i + 1 == N && trig)) {
        if (tid == 0) bulk_load(abuf[0], packed + (size_t)(i + 1) * row_stride, rowbytes, &bars[0]);
        infl0 = true;
    }

    R x[D];
    {
        V2<R> unused[D];
        start_point<R, D>(P, i, m, x, unused, false);
    }
    const bool damp = P.q_damp != 0.0;
    const R qh = (R)(0.5 * P.q_damp);
    const R lw0 = damp ? damp_logw<R, D>(qh, x) : (R)0;  // log w(X_i^i)
    R sum = 0, comp = 0, gN = 0;
    unsigned long long hits = 0;
    V2<R>* mypw = pw + tid;
    const R dt = (R)P.dt;

    for (int j = i; j < N; ++j) {
        const int buf = (j - i) & 1, row = j + 1;
        const bool use_series = row < N || trig;
        const int nrow = row + 1;
        if (nrow < N || (nrow == N && trig)) {
            // the other buffer was last read at the previous step, which
            // ended with a block barrier
            if (tid == 0) {
                fence_proxy_async_smem();
                bulk_load((buf ? abuf[0] : abuf[1]), packed + (size_t)nrow * row_stride, rowbytes, &bars[buf ^ 1]);
            }
            if (buf) infl0 = true;
            else infl1 = true;
        }
        R z[D], x1[D];
        normals<R, D>(P, i, (uint32_t)m, j, z);
        euler<R, D>(P, x, z, x1);
        R y;
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
                return;
            }
            V2<R> zz[D];
#pragma unroll
            for (int l = 0; l < D; ++l) zz[l] = nu_phase<R>(P, x1[l]);
            fill_powers<R, D>(mypw, K1, BS, zz);
            y = series<R, D>((buf ? abuf[1] : abuf[0]), tab, first, nGp, mypw, K1, BS);
            if (damp && row < N) y = undamp<R>(y, damp_logw<R, D>(qh, x1));  // y = ybar^q w(X_{j+1})
            if (row < N && P.clamp_L > 0.0) {
                const R L = (R)P.clamp_L;
                if (y > L) {
                    y = L;
                    ++hits;
                } else if (y < -L) {
                    y = -L;
                    ++hits;
                }
            }
        } else {
            y = term_g<R, D>(P, x1);
        }
        if (row == N) gN = y;
        // S += f(t_j, X_j, y_{j+1}) dt, compensated
        const R term = drv_f<R, D>(P, j, x, y) * dt;
        const R yk = term - comp;
        const R tk = sum + yk;
        comp = (tk - sum) - yk;
        sum = tk;
#pragma unroll
        for (int l = 0; l < D; ++l) x[l] = x1[l];
        __syncthreads();
    }
    // S^q_i = [g(X_N) + sum_j f dt] / w(X_i^i), eq. (Sqi:bar:M)
    const R Sv = damp ? (gN + sum) * (R)exp((double)-lw0) : gN + sum;
    unsigned long long bad = 0;
    if (active) {
        if (in_bounds(P, i - i_lo >= 0 && i - i_lo < P.N)) S[(size_t)(i - i_lo) * (size_t)P.M + (size_t)m] = Sv;
        if (!isfinite(Sv)) bad = 1;
    } else {
        hits = 0;
    }
    hits = warp_sum(hits);
    bad = warp_sum(bad);
    if ((tid & 31) == 0) {
        if (hits) atomicAdd(&counters[CNT_CLAMP], hits);
        if (bad) atomicAdd(&counters[CNT_NONFINITE], bad);
    }
}

// --------------------------------------------------------- projection kernel
template <typename R, int D>
__device__ __forceinline__ void start_phases(const QrParams& P, int i, long long m, V2<R> (&ph)[D])
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

template <typename R, int D, int BS, bool TG>
__global__ void __launch_bounds__(BS) k_project(const __grid_constant__ QrParams P, const GEntry* __restrict__ gtab,
                                                const uint8_t* __restrict__ gfirst, const R* __restrict__ S,
                                                double2* __restrict__ partial, int i_lo, int KT)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int W = BS / 32;
    const int nGp = P.nGp, K1 = P.K1;
    size_t off = 0;
    GEntry* stab = reinterpret_cast<GEntry*>(smem + off);
    if (!TG) off += align16((size_t)nGp * sizeof(GEntry));
    uint8_t* sfirst = smem + off;
    if (!TG) off += align16((size_t)nGp);
    const GEntry* tab = TG ? gtab : stab;
    const uint8_t* first = TG ? gfirst : sfirst;
    V2<R>* pw = reinterpret_cast<V2<R>*>(smem + off);
    off += (size_t)D * K1 * BS * sizeof(V2<R>);
    V2<R>* acc = reinterpret_cast<V2<R>*>(smem + off);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nc = P.c_hi - P.c_lo;  // the context's chunks
    const int i = i_lo + (int)(blockIdx.x / nc);
    const int ch = P.c_lo + (int)(blockIdx.x % nc);
    if (!TG)
        for (int e = tid; e < nGp; e += BS) {
            stab[e] = gtab[e];
            sfirst[e] = gfirst[e];
        }
    V2<R>* mypw = pw + tid;
    const int rounds = P.chunk / BS;

    for (int e0 = 0; e0 < nGp; e0 += KT) {
        const int e1 = min(nGp, e0 + KT);
        for (int t = tid; t < W * KT; t += BS) acc[t] = mk2<R>((R)0, (R)0);
        __syncthreads();
        for (int r = 0; r < rounds; ++r) {
            const long long m = (long long)ch * P.chunk + (long long)r * BS + tid;
            const bool active = m < P.M;
            const R Sv = active && in_bounds(P, i - i_lo >= 0 && i - i_lo < P.N)
                             ? S[(size_t)(i - i_lo) * (size_t)P.M + (size_t)m]
                             : (R)0;
            V2<R> ph[D];
            start_phases<R, D>(P, i, active ? m : 0, ph);
            fill_powers<R, D>(mypw, K1, BS, ph);
            V2<R> b[D];
            V2<R>* wacc = acc + warp * KT - e0;
            for (int e = e0; e < e1; ++e) {
                basis_step<R, D>(b, tab[e], e == e0 ? 0 : first[e], mypw, K1, BS);
                R cr = Sv * b[D - 1].x, ci = -Sv * b[D - 1].y;  // S conj(phi_k(U))
                cr = warp_sum(cr);
                ci = warp_sum(ci);
                if (lane == 0) {
                    V2<R> a = wacc[e];
                    a.x += cr;
                    a.y += ci;
                    wacc[e] = a;
                }
            }
        }
        __syncthreads();
        for (int e = e0 + tid; e < e1; e += BS) {
            double sx = 0.0, sy = 0.0;
            for (int w = 0; w < W; ++w) {
                const V2<R> a = acc[w * KT + (e - e0)];
                sx += (double)a.x;
                sy += (double)a.y;
            }
            if (in_bounds(P, i - i_lo >= 0 && i - i_lo < P.N && ch >= 0 && ch < P.n_chunks && e < nGp))
                partial[((size_t)(i - i_lo) * P.n_chunks + ch) * nGp + e] = make_double2(sx, sy);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------- reduction kernel
// the deterministic cross-chunk sum of the partials of rows i_lo.. (partial
// rows relative to i_lo): chunks summed in order within each of the
// kShardGroups groups, then the groups in order
template <typename R>
__global__ void k_reduce(const __grid_constant__ QrParams P, const double2* __restrict__ partial,
                         double2* __restrict__ alpha, int nG, int zero_idx, V2<R>* __restrict__ packed,
                         long long row_stride, int i_lo, int i_hi, unsigned long long* __restrict__ counters)
{
    const int nGp = P.nGp;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)(i_hi - i_lo) * nGp;
    double diff = 0.0;
    if (idx < total) {
        const int ii = (int)(idx / nGp), e = (int)(idx % nGp), i = i_lo + ii;
        double sx, sy;
        chunk_sum2(partial + (size_t)ii * P.n_chunks * nGp + e, P.n_chunks, nGp, sx, sy);
        finish_coef<R>(P, sx, sy, e, i, nG, zero_idx, alpha, packed, row_stride, diff);
    }
    reduce_residual(diff, &counters[CNT_RESID]);
}

// the group sums of the groups [g_lo, g_hi) of rows i_lo.., from the chunk
// partials of those groups: gsum[g][row][e] (rows absolute, N per group)
__global__ void k_group_sums(const __grid_constant__ QrParams P, const double2* __restrict__ partial,
                             double2* __restrict__ gsum, int g_lo, int g_hi, int i_lo, int i_hi)
{
    const int nGp = P.nGp, rows = i_hi - i_lo;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)(g_hi - g_lo) * rows * nGp) return;
    const int e = (int)(idx % nGp), ii = (int)((idx / nGp) % rows), g = g_lo + (int)(idx / ((long long)nGp * rows));
    const double2* p = partial + (size_t)ii * P.n_chunks * nGp + e;
    double gx = 0.0, gy = 0.0;
    for (int c = group_chunk(g, P.n_chunks); c < group_chunk(g + 1, P.n_chunks); ++c) {
        const double2 v = p[(size_t)c * nGp];
        gx += v.x;
        gy += v.y;
    }
    gsum[((size_t)g * P.N + (i_lo + ii)) * nGp + e] = make_double2(gx, gy);
}

// the reduction from the group sums of every group: the same operations, in
// the same order, as k_reduce from the partials
template <typename R>
__global__ void k_reduce_groups(const __grid_constant__ QrParams P, const double2* __restrict__ gsum,
                                double2* __restrict__ alpha, int nG, int zero_idx, V2<R>* __restrict__ packed,
                                long long row_stride, int i_lo, int i_hi, unsigned long long* __restrict__ counters)
{
    const int nGp = P.nGp;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)(i_hi - i_lo) * nGp;
    double diff = 0.0;
    if (idx < total) {
        const int ii = (int)(idx / nGp), e = (int)(idx % nGp), i = i_lo + ii;
        double sx = 0.0, sy = 0.0;
        for (int g = 0; g < kShardGroups; ++g) {
            const double2 v = gsum[((size_t)g * P.N + i) * nGp + e];
            sx += v.x;
            sy += v.y;
        }
        finish_coef<R>(P, sx, sy, e, i, nG, zero_idx, alpha, packed, row_stride, diff);
    }
    reduce_residual(diff, &counters[CNT_RESID]);
}

// Cosine basis (Lemma ortho:dim1) through the unfolded Fourier set: with
// v = F(x)/2, C_k(F(x)) = prod_l w_l cos(2 pi k_l v_l) expands over the sign
// orbit of k, so a cosine series is the Z^d series with the real, sign-
// symmetric coefficients c_m = a_|m| prod_{m_l != 0} (w/2), evaluated at the
// half-angle phases, and the Monte-Carlo cosine projection of eq. (Aqi:bar:M)
// is, in the same coordinates, the average of Re alpha over the sign orbit:
//     c_m = 2^-d'(m) sum_{s in orbit(m)} Re alpha_s.
// Reads the raw projections of rows [i_lo, i_hi), writes c into alpha and the
// residual max(|c - c_old|) into counters[CNT_RESID].
__global__ void k_sym_cos(const double2* __restrict__ raw, double2* __restrict__ alpha, int nG,
                          const int* __restrict__ orb_off, const int* __restrict__ orb_idx, int i_lo, int i_hi,
                          unsigned long long* __restrict__ counters)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)(i_hi - i_lo) * nG;
    double diff = 0.0;
    if (idx < total) {
        const int i = i_lo + (int)(idx / nG), e = (int)(idx % nG);
        const double2* r = raw + (size_t)i * nG;
        const int a = orb_off[e], b = orb_off[e + 1];
        double s = 0.0;
        for (int t = a; t < b; ++t) s += r[orb_idx[t]].x;
        s /= (double)(b - a);
        double2* row = alpha + (size_t)i * nG;
        const double2 old = row[e];
        diff = hypot(s - old.x, old.y);
        row[e] = make_double2(s, 0.0);
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) diff = fmax(diff, __shfl_xor_sync(0xffffffffu, diff, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = diff;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mx = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
        atomicMax(&counters[CNT_RESID], (unsigned long long)__double_as_longlong(mx));
    }
}

template <typename R>
__global__ void k_pack(const double2* __restrict__ alpha, int nG, int zero_idx, int nGp, V2<R>* __restrict__ packed,
                       long long row_stride, int rows)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)rows * nGp) return;
    const int i = (int)(idx / nGp), e = (int)(idx % nGp);
    const double2 a = alpha[(size_t)i * nG + zero_idx + e];
    packed[(size_t)i * row_stride + e] = e == 0 ? mk2<R>((R)a.x, (R)0) : mk2<R>((R)(2.0 * a.x), (R)(2.0 * a.y));
}

// ------------------------------------------------------------ evaluation
template <typename R, int D, int BS, bool TG>
__global__ void __launch_bounds__(BS) k_eval(const __grid_constant__ QrParams P, const GEntry* __restrict__ gtab,
                                             const uint8_t* __restrict__ gfirst, const V2<R>* __restrict__ crow,
                                             const double* __restrict__ xs, long long n, double* __restrict__ ys,
                                             int use_g)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int nGp = P.nGp, K1 = P.K1;
    size_t off = 0;
    GEntry* stab = reinterpret_cast<GEntry*>(smem + off);
    if (!TG) off += align16((size_t)nGp * sizeof(GEntry));
    uint8_t* sfirst = smem + off;
    if (!TG) off += align16((size_t)nGp);
    const GEntry* tab = TG ? gtab : stab;
    const uint8_t* first = TG ? gfirst : sfirst;
    V2<R>* coef = reinterpret_cast<V2<R>*>(smem + off);
    off += align16((size_t)nGp * sizeof(V2<R>));
    V2<R>* pw = reinterpret_cast<V2<R>*>(smem + off);
    const int tid = threadIdx.x;
    for (int e = tid; e < nGp; e += BS) {
        if (!TG) {
            stab[e] = gtab[e];
            sfirst[e] = gfirst[e];
        }
        if (!use_g) coef[e] = crow[e];
    }
    __syncthreads();
    const long long p = (long long)blockIdx.x * BS + tid;
    if (p >= n) return;
    R x[D];
#pragma unroll
    for (int l = 0; l < D; ++l) x[l] = (R)xs[p * D + l];
    if (use_g) {
        ys[p] = (double)term_g<R, D>(P, x);
        return;
    }
    V2<R> zz[D];
#pragma unroll
    for (int l = 0; l < D; ++l) zz[l] = nu_phase<R>(P, x[l]);
    fill_powers<R, D>(pw + tid, K1, BS, zz);
    ys[p] = (double)series<R, D>(coef, tab, first, nGp, pw + tid, K1, BS);
}

// ------------------------------------------------------------ test hooks
__global__ void k_philox(const uint32_t* __restrict__ ck, long long n, uint32_t* __restrict__ out)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const uint32_t* a = ck + 6 * t;
    uint4 r = philox4x32_10(make_uint4(a[0], a[1], a[2], a[3]), make_uint2(a[4], a[5]));
    out[4 * t + 0] = r.x;
    out[4 * t + 1] = r.y;
    out[4 * t + 2] = r.z;
    out[4 * t + 3] = r.w;
}

template <typename R, int D>
__global__ void k_sample(const __grid_constant__ QrParams P, int i, long long m0, long long n, int j, double* u,
                         double* x, double* z)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const long long m = m0 + t;
    uint64_t ni[D];
    start_ints<D>(P, i, (uint32_t)m, ni);
    R zz[D];
    normals<R, D>(P, i, (uint32_t)m, j, zz);
#pragma unroll
    for (int l = 0; l < D; ++l) {
        if (u) u[t * D + l] = u_of(ni[l]);
        if (x) x[t * D + l] = (double)nu_icdf<R>(P, ni[l]);
        if (z) z[t * D + l] = (double)zz[l];
    }
}

// test points: X = F^{-1}(U), U from the TEST tag (counter j = 0xffffffff)
template <int D>
__global__ void k_test_points(const __grid_constant__ QrParams P, int i, long long n, double* x)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const uint2 key = make_uint2(P.key0, P.key1);
#pragma unroll
    for (int c = 0; 2 * c < D; ++c) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)t, (uint32_t)c, 0xffffffffu, ctr_hi(P.instance, QR_TAG_TEST, i)), key);
        x[t * D + 2 * c] = nu_icdf<double>(P, u52(r.x, r.y));
        if (2 * c + 1 < D) x[t * D + 2 * c + 1] = nu_icdf<double>(P, u52(r.z, r.w));
    }
}

template <int D>
static cudaError_t test_points_t(const QrParams& P, int i, long long n, double* x, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_test_points<D><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(P, i, n, x);
    return cudaGetLastError();
}

// ------------------------------------------------------------ launchers
constexpr int kBS32 = 256, kBS64 = 128;

// bytes of the index table in shared memory (none when it stays in global memory)
static size_t tab_smem(const QrParams& P, bool tg)
{
    return tg ? 0 : align16((size_t)P.nGp * sizeof(GEntry)) + align16((size_t)P.nGp);
}

template <typename R>
static size_t paths_smem(const QrParams& P, long long row_stride, int D, int BS, bool tg)
{
    return tab_smem(P, tg) + 2 * (size_t)row_stride * sizeof(V2<R>) + (size_t)D * P.K1 * BS * sizeof(V2<R>) + 16;
}

template <typename R, int D, int BS, bool TG>
static cudaError_t paths_bs(const QrParams& P, const GEntry* tab, const uint8_t* first, const void* packed,
                            long long row_stride, void* S, int i_lo, int i_hi, unsigned long long* counters,
                            unsigned* status, cudaStream_t st)
{
    const size_t sm = paths_smem<R>(P, row_stride, D, BS, TG);
    if (sm > 227 * 1024) return cudaErrorInvalidConfiguration;
    auto kern = k_paths<R, D, BS, TG>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    // the paths of the context's chunk range (chunks are multiples of BS)
    const int tiles = (int)((shard_m_hi(P) - shard_m_lo(P) + BS - 1) / BS);
    const long long blocks = (long long)tiles * (i_hi - i_lo);
    if (blocks <= 0) return cudaSuccess;
    kern<<<(unsigned)blocks, BS, sm, st>>>(P, tab, first, static_cast<const V2<R>*>(packed), row_stride,
                                           static_cast<R*>(S), i_lo, tiles, counters, status);
    return cudaGetLastError();
}

// FP32 runs 256-thread blocks when their power tables fit in shared memory,
// else 128 (long one-dimensional sets); FP64 always 128; the index table
// moves to global memory only when nothing else fits
template <typename R, int D>
static cudaError_t paths_t(const QrParams& P, const GEntry* tab, const uint8_t* first, const void* packed,
                           long long row_stride, void* S, int i_lo, int i_hi, unsigned long long* counters,
                           unsigned* status, cudaStream_t st)
{
    constexpr size_t cap = 227 * 1024;
    if (sizeof(R) == 4 && paths_smem<R>(P, row_stride, D, kBS32, false) <= cap)
        return paths_bs<R, D, kBS32, false>(P, tab, first, packed, row_stride, S, i_lo, i_hi, counters, status, st);
    if (paths_smem<R>(P, row_stride, D, kBS64, false) <= cap)
        return paths_bs<R, D, kBS64, false>(P, tab, first, packed, row_stride, S, i_lo, i_hi, counters, status, st);
    return paths_bs<R, D, kBS64, true>(P, tab, first, packed, row_stride, S, i_lo, i_hi, counters, status, st);
}

template <typename R, int D, int BS, bool TG>
static cudaError_t project_bs(const QrParams& P, const GEntry* tab, const uint8_t* first, const void* S,
                              double2* partial, int i_lo, int i_hi, cudaStream_t st)
{
    constexpr int W = BS / 32;
    const size_t base = tab_smem(P, TG) + (size_t)D * P.K1 * BS * sizeof(V2<R>);
    const size_t cap = 227 * 1024;
    if (base + W * sizeof(V2<R>) > cap) return cudaErrorInvalidConfiguration;
    int KT = (int)((cap - base) / (W * sizeof(V2<R>)));
    if (KT > P.nGp) KT = P.nGp;
    const size_t sm = base + (size_t)W * KT * sizeof(V2<R>);
    auto kern = k_project<R, D, BS, TG>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const long long blocks = (long long)(P.c_hi - P.c_lo) * (i_hi - i_lo);
    if (blocks <= 0) return cudaSuccess;
    kern<<<(unsigned)blocks, BS, sm, st>>>(P, tab, first, static_cast<const R*>(S), partial, i_lo, KT);
    return cudaGetLastError();
}

template <typename R, int D>
static cudaError_t project_t(const QrParams& P, const GEntry* tab, const uint8_t* first, const void* S,
                             double2* partial, int i_lo, int i_hi, cudaStream_t st)
{
    constexpr size_t cap = 227 * 1024;
    // room for at least 64 coefficients per pass besides the table and the power tables
    auto fits = [&](int bs, bool tg) {
        return tab_smem(P, tg) + (size_t)D * P.K1 * bs * sizeof(V2<R>) + (bs / 32) * 64 * sizeof(V2<R>) <= cap;
    };
    if (sizeof(R) == 4 && fits(kBS32, false)) return project_bs<R, D, kBS32, false>(P, tab, first, S, partial, i_lo, i_hi, st);
    if (fits(kBS64, false)) return project_bs<R, D, kBS64, false>(P, tab, first, S, partial, i_lo, i_hi, st);
    return project_bs<R, D, kBS64, true>(P, tab, first, S, partial, i_lo, i_hi, st);
}

template <typename R, int D, bool TG>
static cudaError_t eval_bs(const QrParams& P, const GEntry* tab, const uint8_t* first, const void* row,
                           const double* x, long long n, double* y, int use_g, cudaStream_t st)
{
    constexpr int BS = 128;
    const size_t sm = tab_smem(P, TG) + align16((size_t)P.nGp * sizeof(V2<R>)) + (size_t)D * P.K1 * BS * sizeof(V2<R>);
    if (sm > 227 * 1024) return cudaErrorInvalidConfiguration;
    auto kern = k_eval<R, D, BS, TG>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    if (n <= 0) return cudaSuccess;
    kern<<<(unsigned)((n + BS - 1) / BS), BS, sm, st>>>(P, tab, first, static_cast<const V2<R>*>(row), x, n, y,
                                                         use_g);
    return cudaGetLastError();
}

template <typename R, int D>
static cudaError_t eval_t(const QrParams& P, const GEntry* tab, const uint8_t* first, const void* row,
                          const double* x, long long n, double* y, int use_g, cudaStream_t st)
{
    const size_t rest = align16((size_t)P.nGp * sizeof(V2<R>)) + (size_t)D * P.K1 * 128 * sizeof(V2<R>);
    if (tab_smem(P, false) + rest <= 227 * 1024) return eval_bs<R, D, false>(P, tab, first, row, x, n, y, use_g, st);
    return eval_bs<R, D, true>(P, tab, first, row, x, n, y, use_g, st);
}

template <typename R, int D>
static cudaError_t sample_t(const QrParams& P, int i, long long m0, long long n, int j, double* u, double* x,
                            double* z, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_sample<R, D><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(P, i, m0, n, j, u, x, z);
    return cudaGetLastError();
}

#define QR_DISPATCH_D(FN, R, ...)                  \
    switch (P.d) {                                 \
    case 1: return FN<R, 1>(__VA_ARGS__);          \
    case 2: return FN<R, 2>(__VA_ARGS__);          \
    case 3: return FN<R, 3>(__VA_ARGS__);          \
    case 4: return FN<R, 4>(__VA_ARGS__);          \
    case 5: return FN<R, 5>(__VA_ARGS__);          \
    case 6: return FN<R, 6>(__VA_ARGS__);          \
    case 7: return FN<R, 7>(__VA_ARGS__);          \
    case 8: return FN<R, 8>(__VA_ARGS__);          \
    default: return cudaErrorInvalidValue;         \
    }

cudaError_t launch_paths(int prec, const QrParams& P, const GEntry* tab, const uint8_t* first, const void* packed,
                         long long row_stride, void* S, int i_lo, int i_hi, unsigned long long* counters,
                         unsigned* status, cudaStream_t st)
{
    if (prec == QR_FP32) {
        QR_DISPATCH_D(paths_t, float, P, tab, first, packed, row_stride, S, i_lo, i_hi, counters, status, st)
    }
    QR_DISPATCH_D(paths_t, double, P, tab, first, packed, row_stride, S, i_lo, i_hi, counters, status, st)
}

cudaError_t launch_project(int prec, const QrParams& P, const GEntry* tab, const uint8_t* first, const void* S,
                           double2* partial, int i_lo, int i_hi, cudaStream_t st)
{
    if (prec == QR_FP32) {
        QR_DISPATCH_D(project_t, float, P, tab, first, S, partial, i_lo, i_hi, st)
    }
    QR_DISPATCH_D(project_t, double, P, tab, first, S, partial, i_lo, i_hi, st)
}

cudaError_t launch_reduce(int prec, const QrParams& P, const double2* partial, double2* alpha, int nG, int zero_idx,
                          void* packed, long long row_stride, int i_lo, int i_hi, unsigned long long* counters,
                          cudaStream_t st)
{
    const long long total = (long long)(i_hi - i_lo) * P.nGp;
    if (total <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    if (prec == QR_FP32)
        k_reduce<float><<<blocks, 256, 0, st>>>(P, partial, alpha, nG, zero_idx, static_cast<float2*>(packed),
                                                row_stride, i_lo, i_hi, counters);
    else
        k_reduce<double><<<blocks, 256, 0, st>>>(P, partial, alpha, nG, zero_idx, static_cast<double2*>(packed),
                                                 row_stride, i_lo, i_hi, counters);
    return cudaGetLastError();
}

cudaError_t launch_group_sums(const QrParams& P, const double2* partial, double2* gsum, int g_lo, int g_hi, int i_lo,
                              int i_hi, cudaStream_t st)
{
    const long long total = (long long)(g_hi - g_lo) * (i_hi - i_lo) * P.nGp;
    if (total <= 0) return cudaSuccess;
    k_group_sums<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(P, partial, gsum, g_lo, g_hi, i_lo, i_hi);
    return cudaGetLastError();
}

cudaError_t launch_reduce_groups(int prec, const QrParams& P, const double2* gsum, double2* alpha, int nG, int zero_idx,
                                 void* packed, long long row_stride, int i_lo, int i_hi,
                                 unsigned long long* counters, cudaStream_t st)
{
    const long long total = (long long)(i_hi - i_lo) * P.nGp;
    if (total <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    if (prec == QR_FP32)
        k_reduce_groups<float><<<blocks, 256, 0, st>>>(P, gsum, alpha, nG, zero_idx, static_cast<float2*>(packed),
                                                       row_stride, i_lo, i_hi, counters);
    else
        k_reduce_groups<double><<<blocks, 256, 0, st>>>(P, gsum, alpha, nG, zero_idx, static_cast<double2*>(packed),
                                                        row_stride, i_lo, i_hi, counters);
    return cudaGetLastError();
}

cudaError_t launch_pack(int prec, const QrParams& P, const double2* alpha, int nG, int zero_idx, void* packed,
                        long long row_stride, int rows, cudaStream_t st)
{
    const long long total = (long long)rows * P.nGp;
    if (total <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    if (prec == QR_FP32)
        k_pack<float><<<blocks, 256, 0, st>>>(alpha, nG, zero_idx, P.nGp, static_cast<float2*>(packed), row_stride,
                                              rows);
    else
        k_pack<double><<<blocks, 256, 0, st>>>(alpha, nG, zero_idx, P.nGp, static_cast<double2*>(packed), row_stride,
                                               rows);
    return cudaGetLastError();
}

cudaError_t launch_eval(int prec, const QrParams& P, const GEntry* tab, const uint8_t* first, const void* packed_row,
                        const double* x, long long n, double* y, int use_g, cudaStream_t st)
{
    if (prec == QR_FP32) {
        QR_DISPATCH_D(eval_t, float, P, tab, first, packed_row, x, n, y, use_g, st)
    }
    QR_DISPATCH_D(eval_t, double, P, tab, first, packed_row, x, n, y, use_g, st)
}

cudaError_t launch_test_points(const QrParams& P, int i, long long n, double* x, cudaStream_t st)
{
    switch (P.d) {
    case 1: return test_points_t<1>(P, i, n, x, st);
    case 2: return test_points_t<2>(P, i, n, x, st);
    case 3: return test_points_t<3>(P, i, n, x, st);
    case 4: return test_points_t<4>(P, i, n, x, st);
    case 5: return test_points_t<5>(P, i, n, x, st);
    case 6: return test_points_t<6>(P, i, n, x, st);
    case 7: return test_points_t<7>(P, i, n, x, st);
    case 8: return test_points_t<8>(P, i, n, x, st);
    case 9: return test_points_t<9>(P, i, n, x, st);
    case 10: return test_points_t<10>(P, i, n, x, st);
    case 11: return test_points_t<11>(P, i, n, x, st);
    case 12: return test_points_t<12>(P, i, n, x, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_philox(const uint32_t* ctr_key, long long n, uint32_t* out, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_philox<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ctr_key, n, out);
    return cudaGetLastError();
}

cudaError_t launch_sample(int prec, const QrParams& P, int i, long long m0, long long n, int j, double* u, double* x,
                          double* z, cudaStream_t st)
{
    if (prec == QR_FP32) {
        QR_DISPATCH_D(sample_t, float, P, i, m0, n, j, u, x, z, st)
    }
    QR_DISPATCH_D(sample_t, double, P, i, m0, n, j, u, x, z, st)
}

cudaError_t launch_sym_cos(const double2* raw, double2* alpha, int nG, const int* orb_off, const int* orb_idx,
                           int i_lo, int i_hi, unsigned long long* counters, cudaStream_t st)
{
    const long long total = (long long)(i_hi - i_lo) * nG;
    if (total <= 0) return cudaSuccess;
    k_sym_cos<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(raw, alpha, nG, orb_off, orb_idx, i_lo, i_hi,
                                                               counters);
    return cudaGetLastError();
}

// Test of the bounded waits: one arrival with 16 bytes of expected
// transaction and no copy behind it, so the barrier phase never completes;
// the bounded wait gives up (~2^31 cycles), the status word records the
// timeout and the kernel returns. No copy is in flight when it exits.
__global__ void k_wait_selftest(unsigned* __restrict__ status)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0)
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bar)), "r"(16u)
                     : "memory");
    __syncthreads();
    const bool ok = mbar_wait(&bar, 0u);
    if (!__syncthreads_and(ok) && threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
}

cudaError_t launch_wait_selftest(unsigned* status, cudaStream_t st)
{
    k_wait_selftest<<<1, 32, 0, st>>>(status);
    return cudaGetLastError();
}

}  // namespace qr
