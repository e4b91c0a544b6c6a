// qr_api.cu -- host side of libqrmc: argument checking, the index set Gamma,
// the coefficient table, device state and the C-ABI of include/qr.h.
#include <algorithm>
#include <map>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <complex>
#include <functional>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "qr_batch.h"
#include "qr_cosine.h"
#include "qr_group.h"
#include "qr_fast.h"
#include "qr_internal.h"

using namespace qr;

struct qr_ctx {
    int d = 0, N = 0, prec = QR_FP64;
    int nG = 0, nGp = 0, zero_idx = 0, kmax = 0;
    std::vector<int> k;  // nG * d, canonical order
    QrParams P{};
    bool trig_g = false;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    long long row_stride = 0;  // elements of the packed coefficient rows
    size_t elem = 0;           // bytes of one packed coefficient
    GEntry* d_tab = nullptr;
    uint8_t* d_first = nullptr;
    double2* d_alpha = nullptr;  // (N+1) x nG, row N = coefficients of a polynomial g
    void* d_packed = nullptr;    // (N+1) x row_stride
    void* d_S = nullptr;         // N x M responses (float or double)
    double2* d_partial = nullptr;
    unsigned long long* d_counters = nullptr;
    unsigned* d_status = nullptr;
    unsigned long long* h_counters = nullptr;  // pinned
    // tree-layout kernel (compiled for this index set): coefficient rows in
    // traversal order, rebuilt from the master rows after every reduction
    int gkind = 0, gn = 0;
    int tree_slots = 0;
    long long tree_stride = 0;
    void* d_tree = nullptr;
    TreeMap* d_tmap = nullptr;
    int proj_nodes = 0;  // tiled projection kernel compiled for this set
    int* d_perm = nullptr;
    // one problem sharded over ranks by path chunks (qr_shard): this
    // context's rank and world size, and the group sums exchanged per iteration
    int shard_rank = 0, shard_world = 1;
    // the caller's device allocator (qr_opts), NULL: cudaMallocAsync
    void* (*dev_alloc)(size_t, void*, void*) = nullptr;
    void (*dev_free)(void*, void*, void*) = nullptr;
    void* alloc_user = nullptr;
    bool coefs_changed = true;  // by qr_set_coefs since a batch last packed its group blocks
    int fault = QR_FAULT_NONE;  // armed host-side fault (qr_inject_fault), taken once
    double2* d_gsum = nullptr;  // kShardGroups x N x |Gamma_+|
    // cosine basis on N^d (Lemma ortho:dim1), run as the unfolded Z^d set
    // with half-angle phases; raw projections are symmetrised over the sign
    // orbits (CSR over the canonical order) after every reduction
    bool cosine = false;
    // the N^d set Gamma of a cosine context (canonical order) and its maps to
    // the unfolded set: z_of_n[q] = unfolded index of k_q; n_of_z[e] = index
    // in Gamma of |m_e|; zscale[e] = 2^{-d'(m_e)/2} (c_m = a_|m| zscale)
    int nGn = 0;
    std::vector<int> kn, z_of_n, n_of_z;
    std::vector<double> zscale;
    double2* d_alpha_raw = nullptr;
    int* d_orb_off = nullptr;
    int* d_orb_idx = nullptr;
    // or run on Gamma itself by the direct cosine kernels (qr_cosine.cu):
    // real rows of cos_groups groups of 4 packed positions; d_cpos[e] =
    // packed position of entry e (then k == kn, nG == nGn, zero_idx == 0)
    bool cos_direct = false;
    int cos_groups = 0;
    CosGroup* d_cgroups = nullptr;
    uint8_t* d_cflags = nullptr;  // one byte per group: run start, changed prefix coordinate
    int* d_cpos = nullptr;
    // one Picard iteration captured as a CUDA graph (built on first use when
    // profiling is off and the stream can be captured)
    cudaGraphExec_t graph = nullptr;
    bool graph_failed = false;
    bool profiling = false;
    cudaEvent_t ev[8] = {};
    qr_stats_t stats{};
    std::string err;
};

namespace {

qr_status fail(qr_ctx* c, qr_status s, const std::string& msg)
{
    if (c) c->err = msg;
    return s;
}

qr_status cuda_fail(qr_ctx* c, cudaError_t e, const char* where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    if (c) c->err = m;
    return QR_ECUDA;
}

#define QR_CU(ctx, call)                                    \
    do {                                                    \
        cudaError_t _e = (call);                            \
        if (_e != cudaSuccess) return cuda_fail(ctx, _e, #call); \
    } while (0)

// Gamma of Z^d in canonical (lexicographic) order.
// nonneg: only k in N^d (the index sets of the cosine basis), same order.
void enumerate_gamma(int kind, int d, int n, std::vector<int>& out, bool nonneg = false)
{
    std::vector<int> k(d, 0);
    std::function<void(int, long long, long long)> rec = [&](int l, long long s, long long prod) {
        for (int v = nonneg ? 0 : -n; v <= n; ++v) {
            const long long a = v < 0 ? -v : v;
            long long s2 = s, p2 = prod;
            if (kind == QR_G_LINF) {
                if (a > n) continue;
            } else if (kind == QR_G_L1) {
                s2 = s + a;
                if (s2 > n) continue;
            } else {
                p2 = prod * (a > 1 ? a : 1);
                if (p2 > n) continue;
            }
            k[l] = v;
            if (l + 1 == d)
                out.insert(out.end(), k.begin(), k.end());
            else
                rec(l + 1, s2, p2);
        }
    };
    rec(0, 0, 1);
}

// Tree layout of the half set (mirrors the traversal of qr_tree.cuh): the
// root slot, then for each dimension the subtree of +e_l; a node's slot is
// followed by its extension child and its children in the later dimensions,
// whose + and - subtrees follow each other; +-1 leaf pairs and the mirrored
// chains of the last dimension are pre-combined pairs; the mirrored chains of
// the QR_TREE_PAIR_LEVELS dimensions before it are, per m, a sum subtree A_m
// and a difference subtree B_m of pre-combined coefficients.
//
// A slot is a real-linear form in the coefficient row; it is built from
// "virtual coefficients" v = sum_t f_t alpha_{e_t} (f_t complex), of which
// every traversal position sees one: alpha_k itself or, inside a pair
// chain of dimension l, v(k) + v(k') (A) and i v(k) - i v(k') (B) of the
// enclosing virtual coefficient v, k' = k mirrored in dimension l.
bool build_tree_map(int kind, int d, int n, const std::vector<int>& K, std::vector<TreeMap>& out)
{
    const int nG = (int)(K.size() / d);
    auto key = [&](const std::vector<int>& k) {
        long long h = 0;
        for (int l = 0; l < d; ++l) h = h * 64 + (k[l] + 32);
        return h;
    };
    std::vector<std::pair<long long, int>> idx;
    idx.reserve(nG);
    for (int e = 0; e < nG; ++e) idx.emplace_back(key(std::vector<int>(K.begin() + (size_t)e * d, K.begin() + (size_t)(e + 1) * d)), e);
    std::sort(idx.begin(), idx.end());
    bool ok = true;
    auto find = [&](const std::vector<int>& k) {
        auto it = std::lower_bound(idx.begin(), idx.end(), std::make_pair(key(k), -1));
        if (it != idx.end() && it->first == key(k)) return it->second;
        ok = false;
        return 0;
    };
    using VC = std::vector<std::pair<int, std::complex<double>>>;  // sum f alpha_e
    using CoefFn = std::function<VC(const std::vector<int>&)>;
    const CoefFn plain = [&](const std::vector<int>& k) { return VC{{find(k), 1.0}}; };
    // term `coef * a[ix]` into row h of a slot (merged with a term of the same index)
    auto put = [&](TreeMap& m, int h, int ix, double coef) {
        if (coef == 0.0) return;
        for (int t = 0; t < kTreeTerms; ++t) {
            if (m.c[h][t] != 0.0 && m.i[h][t] == ix) {
                m.c[h][t] += coef;
                return;
            }
            if (m.c[h][t] == 0.0) {
                m.i[h][t] = ix;
                m.c[h][t] = coef;
                return;
            }
        }
        ok = false;  // more terms than a slot holds
    };
    // s Re v and s Im v: Re(f a) = f.re a.re - f.im a.im, Im(f a) = f.re a.im + f.im a.re
    auto re_into = [&](TreeMap& m, int h, const VC& v, double sc) {
        for (const auto& t : v) {
            put(m, h, 2 * t.first, sc * t.second.real());
            put(m, h, 2 * t.first + 1, -sc * t.second.imag());
        }
    };
    auto im_into = [&](TreeMap& m, int h, const VC& v, double sc) {
        for (const auto& t : v) {
            put(m, h, 2 * t.first + 1, sc * t.second.real());
            put(m, h, 2 * t.first, sc * t.second.imag());
        }
    };
    const bool l1 = kind == QR_G_L1;
    auto ext_ok = [&](int S) { return l1 ? S >= 1 : S < n; };
    auto ext_S = [&](int S) { return l1 ? S - 1 : S + 1; };
    auto new_ok = [&](int S) { return l1 ? S >= 1 : true; };
    auto new_S = [&](int S) { return l1 ? S - 1 : 1; };
    auto leaf = [&](int L, int S) { return l1 ? S == 0 : (S == n && L == d - 1); };
    int emitted = 0;
    // a slot holding 2v (the factor 2 of the half-set sum)
    auto single = [&](const VC& v) {
        TreeMap m{};
        re_into(m, 0, v, 2.0);
        im_into(m, 1, v, 2.0);
        out.push_back(m);
        ++emitted;
    };
    // slots (A, C) and (B, E) of v+ w + v- conj(w): T += (A, C) (w.x, w.y) + (B, E) (w.y, w.x),
    // A = a+ + a-, C = a+ - a-, B = b- - b+, E = b+ + b- (a = 2 Re v, b = 2 Im v)
    auto pair = [&](const VC& vp, const VC& vm) {
        TreeMap a{}, b{};
        re_into(a, 0, vp, 2.0);
        re_into(a, 0, vm, 2.0);
        re_into(a, 1, vp, 2.0);
        re_into(a, 1, vm, -2.0);
        im_into(b, 0, vm, 2.0);
        im_into(b, 0, vp, -2.0);
        im_into(b, 1, vp, 2.0);
        im_into(b, 1, vm, 2.0);
        out.push_back(a);
        out.push_back(b);
        emitted += 2;
    };
    // slots of a last-dimension node in state S and its chain of extensions
    auto chain_len = [&](int S) {
        int len = 1;
        while (ext_ok(S)) {
            ++len;
            if (leaf(d - 1, ext_S(S))) break;
            S = ext_S(S);
        }
        return len;
    };
    auto shifted = [](std::vector<int> k, int l, int by) {
        k[l] += by;
        return k;
    };
    // children in the last dimension of a node k in state S
    auto last_children = [&](const std::vector<int>& k, int S, const CoefFn& cf) {
        const int l2 = d - 1;
        if (leaf(l2, new_S(S))) {
            pair(cf(shifted(k, l2, 1)), cf(shifted(k, l2, -1)));
        } else {
            // the mirrored chains k +- m e_{d-1} as pairs, m = 1..len
            const int len = chain_len(new_S(S));
            for (int m = 1; m <= len; ++m) pair(cf(shifted(k, l2, m)), cf(shifted(k, l2, -m)));
        }
    };
    // dimensions in pair form: d-2, d-3, ..., QR_TREE_PAIR_LEVELS of them
    const int nlv = std::max(0, std::min(QR_TREE_PAIR_LEVELS, d - 2));
    auto paired = [&](int l2) { return l2 <= d - 2 && l2 >= d - 1 - nlv; };
    std::function<void(int, int, const std::vector<int>&, const CoefFn&)> node, new_children;
    // the mirrored chains k +- m e_l2 of a node k (k_l2 = 0) whose children
    // there start in state S2: per m the slots of A_m then B_m
    auto pair_chain = [&](int l2, const std::vector<int>& k, int S2, const CoefFn& cf) {
        for (int m = 1, S = S2;; ++m) {
            const std::vector<int> kp = shifted(k, l2, m);
            const CoefFn ca = [&, l2, m](const std::vector<int>& q) {
                VC v = cf(q);
                const VC w = cf(shifted(q, l2, -2 * m));
                v.insert(v.end(), w.begin(), w.end());
                return v;
            };
            const CoefFn cb = [&, l2, m](const std::vector<int>& q) {
                VC v = cf(q), w = cf(shifted(q, l2, -2 * m));
                for (auto& t : v) t.second *= std::complex<double>(0.0, 1.0);
                for (auto& t : w) v.emplace_back(t.first, t.second * std::complex<double>(0.0, -1.0));
                return v;
            };
            single(ca(kp));
            single(cb(kp));
            if (leaf(l2, S)) break;
            if (new_ok(S)) {
                new_children(l2, S, kp, ca);
                new_children(l2, S, kp, cb);
            }
            if (!ext_ok(S)) break;
            S = ext_S(S);
        }
    };
    // children in the dimensions after L of a node k in state S
    new_children = [&](int L, int S, const std::vector<int>& k, const CoefFn& cf) {
        for (int l2 = L + 1; l2 < d; ++l2) {
            if (leaf(l2, new_S(S))) {
                pair(cf(shifted(k, l2, 1)), cf(shifted(k, l2, -1)));
            } else if (l2 == d - 1) {
                last_children(k, S, cf);
            } else if (paired(l2)) {
                pair_chain(l2, k, new_S(S), cf);
            } else {
                node(l2, new_S(S), shifted(k, l2, 1), cf);
                node(l2, new_S(S), shifted(k, l2, -1), cf);
            }
        }
    };
    node = [&](int L, int S, const std::vector<int>& k, const CoefFn& cf) {
        single(cf(k));
        if (ext_ok(S)) {
            const std::vector<int> k2 = shifted(k, L, k[L] > 0 ? 1 : -1);
            if (leaf(L, ext_S(S))) single(cf(k2));
            else node(L, ext_S(S), k2, cf);
        }
        if (new_ok(S)) new_children(L, S, k, cf);
    };
    std::vector<int> zero(d, 0);
    TreeMap r{};
    re_into(r, 0, plain(zero), 1.0);
    im_into(r, 1, plain(zero), 1.0);
    out.push_back(r);
    const int S0 = l1 ? n - 1 : 1;
    for (int l = 0; l < d; ++l) {
        const std::vector<int> k = shifted(zero, l, 1);
        if (leaf(l, S0)) single(plain(k));
        else node(l, S0, k, plain);
    }
    return ok && emitted == (nG - 1) / 2;
}

// Order of the half set in the tiled projection (mirrors FullTree of
// qr_ptree.cuh): depth-first along the chain tree with both signs of every
// new dimension expanded, the +- chains of the last dimension interleaved
// (+1, -1, +2, -2, ...); perm[s] = canonical half-set index (>= 1) of node s.
bool build_proj_perm(int kind, int d, int n, const std::vector<int>& K, int zero_idx, std::vector<int>& perm)
{
    const int nG = (int)(K.size() / d);
    std::vector<std::pair<std::vector<int>, int>> idx;
    for (int e = 0; e < nG; ++e)
        idx.emplace_back(std::vector<int>(K.begin() + (size_t)e * d, K.begin() + (size_t)(e + 1) * d), e);
    std::sort(idx.begin(), idx.end());
    auto find = [&](const std::vector<int>& k) {
        auto it = std::lower_bound(idx.begin(), idx.end(), std::make_pair(k, -1));
        return (it != idx.end() && it->first == k) ? it->second : -1;
    };
    const bool l1 = kind == QR_G_L1;
    bool ok = true;
    std::function<void(int, int, std::vector<int>)> visit = [&](int L, int S, std::vector<int> k) {
        const int e = find(k);
        if (e <= zero_idx) ok = false;
        perm.push_back(e - zero_idx);
        if (l1 ? S >= 1 : S < n) {
            std::vector<int> k2 = k;
            k2[L] += k[L] > 0 ? 1 : -1;
            visit(L, l1 ? S - 1 : S + 1, k2);
        }
        if (l1 ? S >= 1 : true)
            for (int l2 = L + 1; l2 < d; ++l2) {
                const int S2 = l1 ? S - 1 : 1;
                if (l2 == d - 1) {
                    int len = 1;
                    for (int t = S2; l1 ? t >= 1 : t < n; t = l1 ? t - 1 : t + 1) ++len;
                    for (int m = 1; m <= len; ++m)
                        for (int sg : {+1, -1}) {
                            std::vector<int> km = k;
                            km[l2] += sg * m;
                            const int e = find(km);
                            if (e <= zero_idx) ok = false;
                            perm.push_back(e - zero_idx);
                        }
                    continue;
                }
                std::vector<int> kp = k, km = k;
                kp[l2] += 1;
                km[l2] -= 1;
                visit(l2, S2, kp);
                visit(l2, S2, km);
            }
    };
    for (int l = 0; l < d; ++l) {
        std::vector<int> k(d, 0);
        k[l] = 1;
        visit(l, l1 ? n - 1 : 1, k);
    }
    std::vector<int> seen(perm);
    std::sort(seen.begin(), seen.end());
    return ok && (int)perm.size() == (nG - 1) / 2 && std::unique(seen.begin(), seen.end()) == seen.end();
}

// device memory of a context: the caller's allocator when it gave one, else
// stream-ordered allocation on the context's stream
void* ctx_malloc(qr_ctx* c, size_t bytes)
{
    if (c->fault == QR_FAULT_ALLOC) {
        c->fault = QR_FAULT_NONE;
        return nullptr;
    }
    bytes = bytes < 16 ? 16 : bytes;
    if (c->dev_alloc) return c->dev_alloc(bytes, c->stream, c->alloc_user);
    void* q = nullptr;
    return cudaMallocAsync(&q, bytes, c->stream) == cudaSuccess ? q : nullptr;
}

void ctx_free(qr_ctx* c, void* p)
{
    if (!p) return;
    if (c->dev_free)
        c->dev_free(p, c->stream, c->alloc_user);
    else
        cudaFreeAsync(p, c->stream);
}

template <typename T>
qr_status dalloc(qr_ctx* c, T** p, size_t bytes)
{
    void* q = ctx_malloc(c, bytes);
    if (!q) {
        cudaGetLastError();
        return fail(c, QR_ENOMEM, "device allocation failed (" + std::to_string(bytes) + " bytes)");
    }
    *p = static_cast<T*>(q);
    return QR_OK;
}

void release(qr_ctx* c)
{
    if (!c) return;
    if (c->stream || c->own_stream) {
        void* ptrs[] = {c->d_tab,     c->d_first,   c->d_alpha,    c->d_packed,    c->d_S,
                        c->d_partial, c->d_counters, c->d_status,   c->d_tree,      c->d_tmap,
                        c->d_perm,    c->d_alpha_raw, c->d_orb_off, c->d_orb_idx, c->d_cgroups,
                        c->d_cflags,  c->d_cpos,     c->d_gsum};
        cudaStreamSynchronize(c->stream);  // nothing of the context in flight
        for (void* p : ptrs) ctx_free(c, p);
        cudaStreamSynchronize(c->stream);
    }
    if (c->h_counters) cudaFreeHost(c->h_counters);
    for (auto& e : c->ev)
        if (e) cudaEventDestroy(e);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

qr_status check_device_status(qr_ctx* c)
{
    QR_CU(c, cudaMemcpyAsync(c->h_counters, c->d_counters, sizeof(unsigned long long) * CNT_N, cudaMemcpyDeviceToHost,
                             c->stream));
    unsigned st = 0;
    QR_CU(c, cudaMemcpyAsync(&st, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    QR_CU(c, cudaStreamSynchronize(c->stream));
    c->stats.clamp_hits = (long long)c->h_counters[CNT_CLAMP];
    c->stats.nonfinite = (long long)c->h_counters[CNT_NONFINITE];
    if (st & ST_TIMEOUT) return fail(c, QR_ETIMEOUT, "a bounded wait for a bulk copy ran out on the device");
    if (st & ST_BOUNDS) {
        cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream);
        return fail(c, QR_ECUDA, "checked build: a kernel index fell outside its buffer (the access was skipped)");
    }
    return QR_OK;
}

struct Timer {
    qr_ctx* c;
    int slot;
    Timer(qr_ctx* c_, int s) : c(c_), slot(s)
    {
        if (c->profiling) cudaEventRecord(c->ev[2 * slot], c->stream);
    }
    ~Timer()
    {
        if (c->profiling) cudaEventRecord(c->ev[2 * slot + 1], c->stream);
    }
};

void harvest(qr_ctx* c, int slot)
{
    if (!c->profiling) return;
    float ms = 0.f;
    if (cudaEventSynchronize(c->ev[2 * slot + 1]) == cudaSuccess &&
        cudaEventElapsedTime(&ms, c->ev[2 * slot], c->ev[2 * slot + 1]) == cudaSuccess) {
        if (slot == 0) c->stats.ms_paths += ms, c->stats.launches_paths++;
        if (slot == 1) c->stats.ms_project += ms, c->stats.launches_project++;
        if (slot == 2) c->stats.ms_reduce += ms, c->stats.launches_reduce++;
    }
}

cudaError_t pack_tree_rows(qr_ctx* c, int r_lo, int r_hi)
{
    return launch_pack_tree(c->prec, c->d_alpha + (size_t)r_lo * c->nG, c->nG, c->d_tmap, c->tree_slots,
                            static_cast<char*>(c->d_tree) + c->elem * (size_t)r_lo * c->tree_stride, c->tree_stride,
                            r_hi - r_lo, c->stream);
}

// one projection of rows [i_lo, i_hi) from the current packed coefficients
qr_status run_rows_cos(qr_ctx* c, int i_lo, int i_hi)
{
    double* partial = reinterpret_cast<double*>(c->d_partial);
    {
        Timer t(c, 0);
        cudaError_t e = launch_paths_cos(c->prec, c->P, c->d_cflags, c->cos_groups, c->d_packed, c->row_stride,
                                         c->d_S, i_lo, i_hi, c->d_counters, c->d_status, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "path-and-series kernel (cosine)");
    }
    harvest(c, 0);
    {
        Timer t(c, 1);
        cudaError_t e = launch_project_cos(c->prec, c->P, c->d_cgroups, c->d_cflags, c->cos_groups, c->d_S, partial,
                                           c->row_stride, i_lo, i_hi, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "projection kernel (cosine)");
    }
    harvest(c, 1);
    {
        Timer t(c, 2);
        cudaError_t e = launch_reduce_cos(c->prec, c->P, partial, c->d_cpos, c->d_alpha, c->d_packed, c->row_stride,
                                          i_lo, i_hi, c->d_counters, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "reduction kernel (cosine)");
    }
    harvest(c, 2);
    return QR_OK;
}

qr_status run_rows(qr_ctx* c, int i_lo, int i_hi)
{
    QR_CU(c, cudaMemsetAsync(c->d_counters + CNT_RESID, 0, sizeof(unsigned long long), c->stream));
    if (c->cos_direct) return run_rows_cos(c, i_lo, i_hi);
    {
        Timer t(c, 0);
        cudaError_t e = c->tree_slots
                            ? launch_paths_tree(c->prec, c->gkind, c->gn, c->P, c->d_tree, c->tree_stride, c->d_S,
                                                i_lo, i_hi, c->d_counters, c->d_status, c->stream)
                            : launch_paths(c->prec, c->P, c->d_tab, c->d_first, c->d_packed, c->row_stride, c->d_S,
                                           i_lo, i_hi, c->d_counters, c->d_status, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "path-and-series kernel");
    }
    harvest(c, 0);
    {
        Timer t(c, 1);
        cudaError_t e = c->proj_nodes ? launch_project_tree(c->prec, c->gkind, c->gn, c->P, c->d_S, c->d_perm,
                                                            c->d_partial, i_lo, i_hi, c->stream)
                                      : launch_project(c->prec, c->P, c->d_tab, c->d_first, c->d_S, c->d_partial,
                                                       i_lo, i_hi, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "projection kernel");
    }
    harvest(c, 1);
    {
        Timer t(c, 2);
        cudaError_t e;
        if (c->cosine) {
            // raw projections into their own buffer (their residual goes to
            // the spare counter slot), then the sign-orbit average into alpha
            e = launch_reduce(c->prec, c->P, c->d_partial, c->d_alpha_raw, c->nG, c->zero_idx, c->d_packed,
                              c->row_stride, i_lo, i_hi, c->d_counters + (CNT_SPARE - CNT_RESID), c->stream);
            if (e == cudaSuccess)
                e = launch_sym_cos(c->d_alpha_raw, c->d_alpha, c->nG, c->d_orb_off, c->d_orb_idx, i_lo, i_hi,
                                   c->d_counters, c->stream);
            if (e == cudaSuccess)
                e = launch_pack(c->prec, c->P, c->d_alpha + (size_t)i_lo * c->nG, c->nG, c->zero_idx,
                                static_cast<char*>(c->d_packed) + c->elem * (size_t)i_lo * c->row_stride,
                                c->row_stride, i_hi - i_lo, c->stream);
        } else {
            e = launch_reduce(c->prec, c->P, c->d_partial, c->d_alpha, c->nG, c->zero_idx, c->d_packed,
                              c->row_stride, i_lo, i_hi, c->d_counters, c->stream);
        }
        if (e == cudaSuccess && c->tree_slots)
            e = pack_tree_rows(c, i_lo, i_hi);
        if (e != cudaSuccess) return cuda_fail(c, e, "reduction kernel");
    }
    harvest(c, 2);
    return QR_OK;
}

}  // namespace

namespace qr {
bool ctx_view(const qr_ctx* c, CtxView* v)
{
    if (!c || !c->d_packed || !v) return false;
    v->prec = c->prec;
    v->N = c->N;
    v->nG = c->nG;
    v->zero_idx = c->zero_idx;
    v->P = &c->P;
    v->tab = c->d_tab;
    v->first = c->d_first;
    v->stream = c->stream;
    v->device = c->device;
    v->proj_nodes = c->proj_nodes;
    v->gkind = c->gkind;
    v->gn = c->gn;
    v->perm = c->d_perm;
    v->sharded = c->shard_world > 1;
    return true;
}
void ctx_set_error(qr_ctx* c, const char* msg)
{
    if (c) c->err = msg;
}
}  // namespace qr

extern "C" {

const char* qr_status_string(qr_status s)
{
    switch (s) {
    case QR_OK: return "ok";
    case QR_EINVAL: return "invalid argument";
    case QR_ENOMEM: return "out of memory";
    case QR_ECUDA: return "CUDA error";
    case QR_ETIMEOUT: return "device wait timed out";
    case QR_ENONFINITE: return "non-finite responses";
    case QR_ENOTIMPL: return "not implemented";
    }
    return "unknown status";
}

const char* qr_last_error(const qr_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

qr_status qr_init(qr_ctx** out, int d, int N, double T, const qr_nu* nu, const qr_gamma* gamma, const double* b,
                  const double* sigma, const qr_fn* f, const qr_fn* g, const qr_opts* opts)
{
    if (!out) return QR_EINVAL;
    *out = nullptr;
    qr_ctx* c = new (std::nothrow) qr_ctx();
    if (!c) return QR_ENOMEM;
    if (const char* fe = std::getenv("QR_FAULT")) {
        if (!std::strcmp(fe, "alloc")) c->fault = QR_FAULT_ALLOC;
        else if (!std::strcmp(fe, "launch")) c->fault = QR_FAULT_LAUNCH;
        else if (!std::strcmp(fe, "nan")) c->fault = QR_FAULT_NAN;
    }
    auto bail = [&](qr_status s, const std::string& m) {
        // keep the context so that the caller can read the message, but no
        // device state: the caller must still qr_destroy it
        c->err = m;
        *out = c;
        return s;
    };
    if (d < 1 || d > kDMax) return bail(QR_EINVAL, "d must be in [1, 12]");
    if (N < 1 || N > kNMax) return bail(QR_EINVAL, "N must be in [1, 256]");
    if (!(T > 0.0) || !std::isfinite(T)) return bail(QR_EINVAL, "T must be positive");
    if (!nu || !gamma || !b || !sigma || !f || !g) return bail(QR_EINVAL, "null argument");
    if (nu->kind < QR_NU_LOMAX || nu->kind > QR_NU_CAUCHY) return bail(QR_EINVAL, "unknown nu kind");
    if (nu->kind == QR_NU_LOMAX && !(nu->mu > 0.0)) return bail(QR_EINVAL, "nu: mu must be positive");
    if (gamma->kind < QR_G_LINF || gamma->kind > QR_G_HYP_N ||
        gamma->n < ((gamma->kind == QR_G_HYP || gamma->kind == QR_G_HYP_N) ? 1 : 0))
        return bail(QR_EINVAL, "bad index set");
    // N^d sets of the cosine basis run as their unfolding in Z^d:
    // Gamma_F(n) -> |k|_inf <= n, Gamma_T(n) -> |k|_1 <= n, Gamma_H(n) -> prod max(|k_l|, 1) <= n
    const bool cosine = gamma->kind >= QR_G_FULL_N;
    const int zkind = cosine ? gamma->kind - QR_G_FULL_N : gamma->kind;
    qr_opts o{};
    o.M = 1 << 14;
    o.seed = 1;
    o.precision = QR_FP64;
    if (opts) o = *opts;
    if (o.M < 1 || o.M > (1ll << 32)) return bail(QR_EINVAL, "M must be in [1, 2^32]");
    if (o.precision != QR_FP32 && o.precision != QR_FP64) return bail(QR_EINVAL, "unknown precision");
    if (o.instance < 0 || o.instance >= 4096) return bail(QR_EINVAL, "instance must be in [0, 4096)");
    if (!(o.damping_q >= 0.0) || !std::isfinite(o.damping_q)) return bail(QR_EINVAL, "damping_q must be >= 0");
    if (o.uniform_source == QR_U_LATTICE) {
        if (o.lattice_n < 1) return bail(QR_EINVAL, "lattice_n must be positive");
        long long L = 1;
        for (int l = 0; l < d; ++l) L *= o.lattice_n;
        if (L != o.M) return bail(QR_EINVAL, "lattice start points need M = lattice_n^d");
    } else if (o.uniform_source != QR_U_PHILOX) {
        return bail(QR_EINVAL, "unknown uniform source");
    }
    c->d = d;
    c->N = N;
    c->prec = o.precision;

    // index set and coefficient table
    c->cosine = cosine;
    if (o.path_kernel < 0 || o.path_kernel > 2) return bail(QR_EINVAL, "unknown path kernel");
    if (o.path_kernel == 2 && !cosine) return bail(QR_EINVAL, "path_kernel 2 (direct cosine kernels) needs a cosine index set");
    std::vector<GEntry> tab;
    std::vector<uint8_t> first;
    std::vector<CosGroup> cgroups;
    std::vector<uint8_t> cflags;
    std::vector<int> cpos;
    if (cosine) {
        // the direct kernels on Gamma itself, or the unfolded Z^d set on the
        // Fourier kernels: unfolded when asked for (path_kernel 1) or when a
        // compile-time tree kernel covers the unfolded set and its tables fit
        std::vector<int> kn;
        enumerate_gamma(zkind, d, gamma->n, kn, true);
        const int nn = (int)(kn.size() / d);
        long long nz = 0;
        int km = 0;
        for (int q = 0; q < nn; ++q) {
            int dn = 0;
            for (int l = 0; l < d; ++l) {
                dn += kn[(size_t)q * d + l] != 0;
                km = std::max(km, kn[(size_t)q * d + l]);
            }
            nz += 1ll << dn;
        }
        const size_t v2 = o.precision == QR_FP32 ? sizeof(float2) : sizeof(double2);
        const double need = (double)d * (km + 1) * 128 * v2 + 2.0 * (double)((nz + 1) / 2) * v2 + 256;
        const bool unfold_ok = km <= gentry_kmax(d) && need <= 227.0 * 1024;
        c->cos_direct = o.path_kernel == 2 || d > kDMaxFourier ||
                        (o.path_kernel == 0 && (!unfold_ok || zkind == QR_G_HYP || tree_slots(zkind, d, gamma->n) == 0));
        if (c->cos_direct && o.path_kernel == 1)
            return bail(QR_ENOTIMPL, "the unfolded cosine route needs d <= 8 (path_kernel 0 or 2)");
        if (c->cos_direct) {
            c->k = std::move(kn);
            c->kmax = km;
        } else if (!unfold_ok) {
            return bail(QR_ENOTIMPL, "the unfolded set of this cosine index set exceeds the shared memory of the "
                                     "table kernels (path_kernel 2 runs it on the direct kernels)");
        }
    }
    if (c->cos_direct) {
        // runs of Gamma (common k_1..k_{d-1}, k_d = 0, 1, ...) in groups of 4 packed positions
        c->nG = (int)(c->k.size() / d);
        c->nGn = c->nG;
        c->kn = c->k;
        c->zero_idx = 0;
        c->nGp = c->nG;
        if (d > 1 && c->kmax > kCosPrefixMax)
            return bail(QR_ENOTIMPL, "direct cosine kernels: k_l <= 255 is required for d > 1");
        if (c->kmax > 65532) return bail(QR_ENOTIMPL, "direct cosine kernels: k <= 65532 is required");
        cpos.resize(c->nG);
        std::vector<int> prev(d > 1 ? d - 1 : 1, -1);
        for (int e = 0; e < c->nG;) {
            const int* ke = &c->k[(size_t)e * d];
            int len = 0;
            while (e + len < c->nG && std::equal(ke, ke + d - 1, &c->k[(size_t)(e + len) * d])) {
                if (c->k[(size_t)(e + len) * d + d - 1] != len)
                    return bail(QR_ENOTIMPL, "direct cosine kernels: a run of Gamma does not start at k_d = 0");
                cpos[e + len] = 4 * (int)cgroups.size() + len;
                ++len;
            }
            int f = 0;
            if (d > 1 && e > 0)
                while (f < d - 1 && ke[f] == prev[f]) ++f;
            // the kernels step the prefix: coordinate f one up, the later ones back to 0
            bool step_ok = true;
            for (int l = 0; l + 1 < d; ++l) {
                const int want = e == 0 ? 0 : (l < f ? prev[l] : (l == f ? prev[l] + 1 : 0));
                step_ok = step_ok && ke[l] == want;
            }
            if (!step_ok) return bail(QR_ENOTIMPL, "direct cosine kernels: Gamma is not downward closed");
            uint32_t kz = 0, kw = 0, ky = 0;
            for (int l = 0; l + 1 < d; ++l) {
                (l < 4 ? kz : (l < 8 ? kw : ky)) |= (uint32_t)ke[l] << (8 * (l & 3));
                prev[l] = ke[l];
            }
            for (int a0 = 0; a0 < len; a0 += 4) {
                cgroups.push_back(make_uint4((uint32_t)a0, ky, kz, kw));
                cflags.push_back((uint8_t)(a0 == 0 ? 0x80 | (e == 0 ? d - 1 : f) : d - 1));
            }
            e += len;
        }
        while (cgroups.size() % 16) {  // runs of zero coefficients under the last prefix
            uint4 q = cgroups.back();
            q.x = 0;
            cgroups.push_back(q);
            cflags.push_back((uint8_t)(0x80 | (d - 1)));
        }
        c->cos_groups = (int)cgroups.size();
    } else {
        if (d > kDMaxFourier) return bail(QR_ENOTIMPL, "index sets of Z^d need d <= 8");
        enumerate_gamma(zkind, d, gamma->n, c->k);
        if (cosine) {
            const int nz = (int)(c->k.size() / d);
            std::map<std::vector<int>, int> nidx;
            for (int e = 0; e < nz; ++e) {
                std::vector<int> kv(c->k.begin() + (size_t)e * d, c->k.begin() + (size_t)(e + 1) * d);
                bool nonneg = true;
                for (int v : kv) nonneg = nonneg && v >= 0;
                if (nonneg) {
                    nidx[kv] = (int)c->z_of_n.size();
                    c->z_of_n.push_back(e);
                    c->kn.insert(c->kn.end(), kv.begin(), kv.end());
                }
            }
            c->nGn = (int)c->z_of_n.size();
            c->n_of_z.resize(nz);
            c->zscale.resize(nz);
            for (int e = 0; e < nz; ++e) {
                std::vector<int> kv(c->k.begin() + (size_t)e * d, c->k.begin() + (size_t)(e + 1) * d);
                int dn = 0;
                for (int& v : kv) {
                    dn += v != 0;
                    v = v < 0 ? -v : v;
                }
                c->n_of_z[e] = nidx.at(kv);
                c->zscale[e] = std::pow(2.0, -0.5 * dn);
            }
        }
        c->nG = (int)(c->k.size() / d);
        c->zero_idx = (c->nG - 1) / 2;
        for (int l = 0; l < d; ++l)
            if (c->k[(size_t)c->zero_idx * d + l] != 0) return bail(QR_EINVAL, "index set is not symmetric");
        for (int v : c->k) c->kmax = std::max(c->kmax, v < 0 ? -v : v);
        if (c->kmax > gentry_kmax(d))
            return bail(QR_ENOTIMPL, d <= 4 ? "|k_l| <= 32767 is required" : "|k_l| <= 127 is required for d > 4");
        {
            // the table kernels (generic path, projection, evaluation) keep the
            // powers z_l^a, a <= max|k_l|, of every lane in shared memory
            const size_t v2 = o.precision == QR_FP32 ? sizeof(float2) : sizeof(double2);
            const size_t nGp = (size_t)(c->nG - (c->nG - 1) / 2);
            // (the index table itself moves to global memory when it does not fit)
            const size_t need = (size_t)d * (c->kmax + 1) * 128 * v2 + 2 * nGp * v2 + 256;
            if (need > 227 * 1024)
                return bail(QR_ENOTIMPL, "index set too large for the table kernels: " + std::to_string(need / 1024) +
                                             " KB of shared memory per block (limit 227 KB)");
        }
        c->nGp = c->nG - c->zero_idx;
        tab.resize(c->nGp);
        first.assign(c->nGp, 0);
        for (int e = 0; e < c->nGp; ++e) {
            std::memset(tab[e].k8, 0, sizeof(tab[e].k8));
            for (int l = 0; l < d && l < kDMaxFourier; ++l) tab[e].set(d, l, c->k[(size_t)(c->zero_idx + e) * d + l]);
            if (e > 0) {
                int f0 = 0;
                while (f0 < d && tab[e].get(d, f0) == tab[e - 1].get(d, f0)) ++f0;
                first[e] = (uint8_t)f0;
            }
        }
    }

    // problem parameters
    QrParams& P = c->P;
    P.d = d;
    P.half_angle = cosine ? 1 : 0;
    P.q_damp = o.damping_q;
    P.N = N;
    P.nGp = c->nGp;
    P.K1 = c->kmax + 1;
    P.M = o.M;
    P.nu_kind = nu->kind;
    P.mu = nu->kind == QR_NU_LOMAX ? nu->mu : (nu->kind == QR_NU_STUDENT2 ? 2.0 : 1.0);
    P.inv_mu = 1.0 / P.mu;
    P.mu_is3 = nu->kind == QR_NU_LOMAX && nu->mu == 3.0;
    P.T = T;
    P.dt = T / N;
    P.sqdt = std::sqrt(P.dt);
    P.sig_diag = 1;
    for (int l = 0; l < d; ++l) {
        P.b[l] = b[l];
        for (int cc = 0; cc < d; ++cc) {
            P.sig[l * d + cc] = sigma[l * d + cc];
            if (l != cc && sigma[l * d + cc] != 0.0) P.sig_diag = 0;
        }
    }
    P.f_kind = f->kind;
    switch (f->kind) {
    case QR_F_ZERO:
        break;
    case QR_F_LINEAR:
        if (!f->params || f->n_params < 1) return bail(QR_EINVAL, "linear driver needs {lambda}");
        P.f_lam = f->params[0];
        break;
    case QR_F_CUBIC_MANUF: {
        if (!f->params || f->n_params < 1 + d) return bail(QR_EINVAL, "cubic driver needs {a, s_1..s_d}");
        const double a = f->params[0];
        double st2 = 0.0;
        for (int cc = 0; cc < d; ++cc) {
            double v = 0.0;
            for (int l = 0; l < d; ++l) v += sigma[l * d + cc] * f->params[1 + l];
            st2 += v * v;
        }
        for (int l = 0; l < d; ++l) P.f_s[l] = f->params[1 + l];
        P.f_c = a + 0.5 * st2;
        for (int j = 0; j < N; ++j) P.fexp[j] = std::exp(a * (T - j * P.dt));
        break;
    }
    case QR_F_PAPER_MIN:
        if (!f->params || f->n_params < 2) return bail(QR_EINVAL, "paper driver needs {kappa, lambda}");
        P.f_kap = f->params[0];
        P.f_lam = f->params[1];
        for (int j = 0; j < N; ++j) P.fexp[j] = std::exp(P.f_lam * P.f_lam * d * (j * P.dt - T) / 2.0);
        break;
    default:
        return bail(QR_EINVAL, "unknown driver");
    }
    for (int j = 0; j < N; ++j) P.fexp32[j] = (float)P.fexp[j];
    P.g_kind = g->kind;
    if (g->kind == QR_GT_COS) {
        if (!g->params || g->n_params < d) return bail(QR_EINVAL, "cos terminal needs {s_1..s_d}");
        for (int l = 0; l < d; ++l) P.g_s[l] = g->params[l];
    } else if (g->kind == QR_GT_PAPER_SIN) {
        if (!g->params || g->n_params < 2) return bail(QR_EINVAL, "paper terminal needs {kappa, lambda}");
        P.g_kap = g->params[0];
        P.g_lam = g->params[1];
    } else if (g->kind == QR_GT_TRIGPOLY) {
        if (!g->params || g->n_params < 2 * (cosine ? c->nGn : c->nG))
            return bail(QR_EINVAL, "polynomial terminal needs 2|Gamma| values");
        c->trig_g = true;
    } else {
        return bail(QR_EINVAL, "unknown terminal condition");
    }
    P.key0 = (uint32_t)(o.seed & 0xffffffffull);
    P.key1 = (uint32_t)(o.seed >> 32);
    P.instance = o.instance;
    P.clamp_L = o.clamp_L;
    P.lattice_n = o.uniform_source == QR_U_LATTICE ? o.lattice_n : 0;
    const int BS = c->prec == QR_FP32 ? 256 : 128;
    const long long per = (o.M + 256ll * BS - 1) / (256ll * BS);
    P.chunk = (int)(BS * std::max(1ll, per));
    P.n_chunks = (int)((o.M + P.chunk - 1) / P.chunk);
    P.c_lo = 0;
    P.c_hi = P.n_chunks;

    // device state
    if (!o.dev_alloc != !o.dev_free) return bail(QR_EINVAL, "dev_alloc and dev_free go together");
    c->dev_alloc = o.dev_alloc;
    c->dev_free = o.dev_free;
    c->alloc_user = o.alloc_user;
    QR_CU(c, cudaGetDevice(&c->device));
    if (o.stream) {
        c->stream = static_cast<cudaStream_t>(o.stream);
    } else {
        QR_CU(c, cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    }
    if (c->cos_direct) {  // real rows: groups of 4 positions (16 or 32 bytes)
        c->elem = c->prec == QR_FP32 ? sizeof(float) : sizeof(double);
        c->row_stride = 4ll * c->cos_groups;
    } else {
        c->elem = c->prec == QR_FP32 ? sizeof(float2) : sizeof(double2);
        c->row_stride = c->prec == QR_FP32 ? ((c->nGp + 1) & ~1) : c->nGp;  // rows of 16-byte multiples
    }
    qr_status s;
    if ((s = dalloc(c, &c->d_tab, sizeof(GEntry) * tab.size())) != QR_OK) return bail(s, c->err);
    if ((s = dalloc(c, &c->d_first, first.size())) != QR_OK) return bail(s, c->err);
    if ((s = dalloc(c, &c->d_alpha, sizeof(double2) * (size_t)(N + 1) * c->nG)) != QR_OK) return bail(s, c->err);
    if ((s = dalloc(c, &c->d_packed, c->elem * (size_t)(N + 1) * c->row_stride)) != QR_OK) return bail(s, c->err);
    if ((s = dalloc(c, &c->d_S, (c->prec == QR_FP32 ? 4 : 8) * (size_t)N * (size_t)o.M)) != QR_OK)
        return bail(s, c->err);
    const size_t partial_bytes = c->cos_direct ? sizeof(double) * (size_t)N * P.n_chunks * c->row_stride
                                               : sizeof(double2) * (size_t)N * P.n_chunks * c->nGp;
    if ((s = dalloc(c, &c->d_partial, partial_bytes)) != QR_OK) return bail(s, c->err);
    if (c->cos_direct) {
        if ((s = dalloc(c, &c->d_cgroups, sizeof(CosGroup) * cgroups.size())) != QR_OK ||
            (s = dalloc(c, &c->d_cflags, cflags.size())) != QR_OK ||
            (s = dalloc(c, &c->d_cpos, sizeof(int) * cpos.size())) != QR_OK)
            return bail(s, c->err);
    }
    if ((s = dalloc(c, &c->d_counters, sizeof(unsigned long long) * CNT_N)) != QR_OK) return bail(s, c->err);
    if ((s = dalloc(c, &c->d_status, sizeof(unsigned))) != QR_OK) return bail(s, c->err);
    P.check = c->d_status;
    if (cudaMallocHost(&c->h_counters, sizeof(unsigned long long) * CNT_N) != cudaSuccess)
        return bail(QR_ENOMEM, "pinned host allocation failed");
    for (auto& e : c->ev)
        if (cudaEventCreate(&e) != cudaSuccess) return bail(QR_ECUDA, "event creation failed");

    auto cu = [&](cudaError_t e, const char* w) { return e == cudaSuccess ? QR_OK : cuda_fail(c, e, w); };
    if ((!tab.empty() &&
         (s = cu(cudaMemcpyAsync(c->d_tab, tab.data(), sizeof(GEntry) * tab.size(), cudaMemcpyHostToDevice, c->stream),
                 "copy table")) != QR_OK) ||
        (!first.empty() &&
         (s = cu(cudaMemcpyAsync(c->d_first, first.data(), first.size(), cudaMemcpyHostToDevice, c->stream),
                 "copy table")) != QR_OK) ||
        (c->cos_direct &&
         ((s = cu(cudaMemcpyAsync(c->d_cgroups, cgroups.data(), sizeof(CosGroup) * cgroups.size(),
                                  cudaMemcpyHostToDevice, c->stream),
                  "copy groups")) != QR_OK ||
          (s = cu(cudaMemcpyAsync(c->d_cflags, cflags.data(), cflags.size(), cudaMemcpyHostToDevice, c->stream),
                  "copy run flags")) != QR_OK ||
          (s = cu(cudaMemcpyAsync(c->d_cpos, cpos.data(), sizeof(int) * cpos.size(), cudaMemcpyHostToDevice,
                                  c->stream),
                  "copy positions")) != QR_OK ||
          (s = cu(cudaMemsetAsync(c->d_packed, 0, c->elem * (size_t)(N + 1) * c->row_stride, c->stream),
                  "zero packed rows")) != QR_OK)) ||
        (s = cu(cudaMemsetAsync(c->d_alpha, 0, sizeof(double2) * (size_t)(N + 1) * c->nG, c->stream), "zero alpha")) !=
            QR_OK ||
        (s = cu(cudaMemsetAsync(c->d_counters, 0, sizeof(unsigned long long) * CNT_N, c->stream), "zero counters")) !=
            QR_OK ||
        (s = cu(cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream), "zero status")) != QR_OK)
        return bail(s, c->err);
    std::vector<double2> g_unfolded;  // a cosine polynomial g on the unfolded set (lives until the final sync)
    if (c->trig_g) {
        const double2* src = reinterpret_cast<const double2*>(g->params);
        if (c->cos_direct) {
            g_unfolded.resize(c->nG);
            for (int e = 0; e < c->nG; ++e) g_unfolded[e] = make_double2(g->params[2 * e], 0.0);
            src = g_unfolded.data();
        } else if (cosine) {
            g_unfolded.resize(c->nG);
            for (int e = 0; e < c->nG; ++e)
                g_unfolded[e] = make_double2(g->params[2 * c->n_of_z[e]] * c->zscale[e], 0.0);
            src = g_unfolded.data();
        }
        if ((s = cu(cudaMemcpyAsync(c->d_alpha + (size_t)N * c->nG, src, sizeof(double2) * c->nG,
                                    cudaMemcpyHostToDevice, c->stream),
                    "copy terminal polynomial")) != QR_OK)
            return bail(s, c->err);
    }
    if ((s = cu(c->cos_direct
                    ? launch_pack_cos(c->prec, c->d_alpha, c->nG, c->d_cpos, c->d_packed, c->row_stride, N + 1,
                                      c->stream)
                    : launch_pack(c->prec, P, c->d_alpha, c->nG, c->zero_idx, c->d_packed, c->row_stride, N + 1,
                                  c->stream),
                "pack")) != QR_OK)
        return bail(s, c->err);
    c->gkind = zkind;
    c->gn = gamma->n;
    if (o.path_kernel == 0 && zkind != QR_G_HYP && !c->cos_direct) c->tree_slots = tree_slots(zkind, d, gamma->n);
    if (c->tree_slots) {
        std::vector<TreeMap> map;
        if (!build_tree_map(zkind, d, gamma->n, c->k, map) || (int)map.size() != c->tree_slots)
            return bail(QR_ENOTIMPL, "tree layout does not match the compiled kernel");
        c->tree_stride = c->prec == QR_FP32 ? ((c->tree_slots + 1) & ~1) : c->tree_slots;
        if ((s = dalloc(c, &c->d_tmap, sizeof(TreeMap) * map.size())) != QR_OK) return bail(s, c->err);
        if ((s = dalloc(c, &c->d_tree, c->elem * (size_t)(N + 1) * c->tree_stride)) != QR_OK) return bail(s, c->err);
        if ((s = cu(cudaMemcpyAsync(c->d_tmap, map.data(), sizeof(TreeMap) * map.size(), cudaMemcpyHostToDevice,
                                    c->stream),
                    "copy tree map")) != QR_OK ||
            (s = cu(pack_tree_rows(c, 0, N + 1), "pack tree")) != QR_OK)
            return bail(s, c->err);
    }
    if (o.path_kernel == 0 && zkind != QR_G_HYP && !c->cos_direct)
        c->proj_nodes = proj_tree_nodes(zkind, d, gamma->n);
    if (c->proj_nodes) {
        std::vector<int> perm;
        if (!build_proj_perm(zkind, d, gamma->n, c->k, c->zero_idx, perm) || (int)perm.size() != c->proj_nodes)
            return bail(QR_ENOTIMPL, "projection order does not match the compiled kernel");
        if ((s = dalloc(c, &c->d_perm, sizeof(int) * perm.size())) != QR_OK) return bail(s, c->err);
        if ((s = cu(cudaMemcpyAsync(c->d_perm, perm.data(), sizeof(int) * perm.size(), cudaMemcpyHostToDevice,
                                    c->stream),
                    "copy projection order")) != QR_OK)
            return bail(s, c->err);
    }
    if (cosine && !c->cos_direct) {
        std::map<std::vector<int>, int> where;
        for (int e = 0; e < c->nG; ++e) where[std::vector<int>(c->k.begin() + (size_t)e * d, c->k.begin() + (size_t)(e + 1) * d)] = e;
        std::vector<int> off(1, 0), idx;
        for (int e = 0; e < c->nG; ++e) {
            std::vector<int> kv(c->k.begin() + (size_t)e * d, c->k.begin() + (size_t)(e + 1) * d), nz;
            for (int l = 0; l < d; ++l)
                if (kv[l] != 0) nz.push_back(l);
            for (int mask = 0; mask < (1 << nz.size()); ++mask) {
                std::vector<int> f = kv;
                for (size_t t = 0; t < nz.size(); ++t)
                    if (mask >> t & 1) f[nz[t]] = -f[nz[t]];
                auto it = where.find(f);
                if (it == where.end()) return bail(QR_EINVAL, "index set is not closed under sign flips");
                idx.push_back(it->second);
            }
            off.push_back((int)idx.size());
        }
        if ((s = dalloc(c, &c->d_alpha_raw, sizeof(double2) * (size_t)(N + 1) * c->nG)) != QR_OK ||
            (s = dalloc(c, &c->d_orb_off, sizeof(int) * off.size())) != QR_OK ||
            (s = dalloc(c, &c->d_orb_idx, sizeof(int) * idx.size())) != QR_OK)
            return bail(s, c->err);
        if ((s = cu(cudaMemcpyAsync(c->d_orb_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice,
                                    c->stream),
                    "copy orbits")) != QR_OK ||
            (s = cu(cudaMemcpyAsync(c->d_orb_idx, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice,
                                    c->stream),
                    "copy orbits")) != QR_OK ||
            (s = cu(cudaMemsetAsync(c->d_alpha_raw, 0, sizeof(double2) * (size_t)(N + 1) * c->nG, c->stream),
                    "zero raw alpha")) != QR_OK)
            return bail(s, c->err);
    }
    if ((s = cu(cudaStreamSynchronize(c->stream), "init sync")) != QR_OK) return bail(s, c->err);
    *out = c;
    return QR_OK;
}

void qr_destroy(qr_ctx* ctx)
{
    if (!ctx) return;
    release(ctx);
    delete ctx;
}

static bool ready(const qr_ctx* c) { return c && c->d_packed; }

// NVTX range over a host call (shows the enqueue of the iterations on a
// profiler's timeline; no cost when no tool is attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// every packed copy of the master coefficient rows, rebuilt from d_alpha
static qr_status repack_all(qr_ctx* ctx)
{
    ctx->coefs_changed = true;
    if (ctx->cos_direct)
        QR_CU(ctx, launch_pack_cos(ctx->prec, ctx->d_alpha, ctx->nG, ctx->d_cpos, ctx->d_packed, ctx->row_stride,
                                   ctx->N, ctx->stream));
    else
        QR_CU(ctx, launch_pack(ctx->prec, ctx->P, ctx->d_alpha, ctx->nG, ctx->zero_idx, ctx->d_packed,
                               ctx->row_stride, ctx->N, ctx->stream));
    if (ctx->tree_slots) QR_CU(ctx, pack_tree_rows(ctx, 0, ctx->N));
    return QR_OK;
}

// the faults an iteration takes at its start (qr_inject_fault)
static qr_status take_iteration_fault(qr_ctx* ctx)
{
    const int f = ctx->fault;
    if (f == QR_FAULT_LAUNCH) {
        ctx->fault = QR_FAULT_NONE;
        return fail(ctx, QR_ECUDA, "injected launch failure (nothing was launched)");
    }
    if (f == QR_FAULT_NAN) {
        ctx->fault = QR_FAULT_NONE;
        if (ctx->N < 2) return QR_OK;  // no coefficient row is read by a series
        // the k = 0 coefficient of the last row becomes NaN in the master row
        // and every packed copy: every series evaluated at t_{N-1} is NaN
        const int k0 = ctx->cos_direct ? 0 : ctx->zero_idx;
        const double2 bad = make_double2(std::nan(""), 0.0);
        QR_CU(ctx, cudaMemcpyAsync(ctx->d_alpha + (size_t)(ctx->N - 1) * ctx->nG + k0, &bad, sizeof bad,
                                   cudaMemcpyHostToDevice, ctx->stream));
        QR_CU(ctx, cudaStreamSynchronize(ctx->stream));
        return repack_all(ctx);
    }
    return QR_OK;
}

qr_status qr_inject_fault(qr_ctx* ctx, int kind)
{
    if (!ctx || kind < QR_FAULT_NONE || kind > QR_FAULT_NAN) return QR_EINVAL;
    ctx->fault = kind;
    return QR_OK;
}

qr_status qr_picard_step(qr_ctx* ctx, int n_iter, double* residual_out)
{
    if (!ready(ctx)) return QR_EINVAL;
    if (ctx->shard_world > 1)
        return fail(ctx, QR_EINVAL, "qr_picard_step: a sharded context iterates by qr_picard_begin/finish");
    if (n_iter < 0) return fail(ctx, QR_EINVAL, "n_iter must be >= 0");
    NvtxRange range("qr_picard_step");
    if (n_iter > 0) {
        qr_status fs = take_iteration_fault(ctx);
        if (fs != QR_OK) return fs;
    }
    QR_CU(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned), ctx->stream));
    if (!ctx->profiling && !ctx->graph && !ctx->graph_failed && n_iter > 0) {
        // capture one iteration; streams that cannot be captured (the legacy
        // default stream) keep the direct launches
        cudaGraph_t g = nullptr;
        bool ok = ctx->stream != nullptr &&
                  cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            qr_status s = run_rows(ctx, 0, ctx->N);
            cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
            ok = s == QR_OK && e == cudaSuccess && g &&
                 cudaGraphInstantiate(&ctx->graph, g, 0) == cudaSuccess;
            if (g) cudaGraphDestroy(g);
        }
        if (!ok) {
            cudaGetLastError();
            ctx->graph = nullptr;
            ctx->graph_failed = true;
            ctx->err.clear();
        }
    }
    for (int q = 0; q < n_iter; ++q) {
        NvtxRange it_range("picard iteration");
        if (ctx->graph && !ctx->profiling) {
            QR_CU(ctx, cudaGraphLaunch(ctx->graph, ctx->stream));
        } else {
            qr_status s = run_rows(ctx, 0, ctx->N);
            if (s != QR_OK) return s;
        }
        ctx->stats.iterations++;
    }
    const long long nonfinite_before = ctx->stats.nonfinite;
    qr_status s = check_device_status(ctx);
    if (s != QR_OK) return s;
    if (residual_out) {
        unsigned long long bits = ctx->h_counters[CNT_RESID];
        double r;
        std::memcpy(&r, &bits, sizeof r);
        *residual_out = n_iter > 0 ? r : 0.0;
    }
    if (ctx->stats.nonfinite > nonfinite_before) return fail(ctx, QR_ENONFINITE, "non-finite responses");
    return QR_OK;
}

// ------------------------------------------------------------ sharding
qr_status qr_shard_plan(int n_chunks, int rank, int world, int* c_lo, int* c_hi, int* g_lo, int* g_hi)
{
    if (n_chunks < 1 || world < 1 || world > kShardGroups || kShardGroups % world != 0 || rank < 0 || rank >= world)
        return QR_EINVAL;
    const int per = kShardGroups / world;
    const int gl = rank * per, gh = gl + per;
    if (g_lo) *g_lo = gl;
    if (g_hi) *g_hi = gh;
    if (c_lo) *c_lo = group_chunk(gl, n_chunks);
    if (c_hi) *c_hi = group_chunk(gh, n_chunks);
    return QR_OK;
}

qr_status qr_shard(qr_ctx* ctx, int rank, int world)
{
    if (!ready(ctx)) return QR_EINVAL;
    if (ctx->cosine) return fail(ctx, QR_ENOTIMPL, "qr_shard: the cosine basis is not supported");
    int cl = 0, ch = 0;
    if (qr_shard_plan(ctx->P.n_chunks, rank, world, &cl, &ch, nullptr, nullptr) != QR_OK)
        return fail(ctx, QR_EINVAL, "qr_shard: world must divide 8 and 0 <= rank < world");
    if (world > 1 && !ctx->d_gsum) {
        qr_status s = dalloc(ctx, &ctx->d_gsum, sizeof(double2) * kShardGroups * (size_t)ctx->N * ctx->nGp);
        if (s != QR_OK) return s;
        QR_CU(ctx, cudaMemsetAsync(ctx->d_gsum, 0, sizeof(double2) * kShardGroups * (size_t)ctx->N * ctx->nGp,
                                   ctx->stream));
    }
    ctx->P.c_lo = cl;
    ctx->P.c_hi = ch;
    ctx->shard_rank = rank;
    ctx->shard_world = world;
    // the captured iteration has the old chunk range baked in
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
    ctx->graph_failed = false;
    return QR_OK;
}

qr_status qr_shard_groups(const qr_ctx* ctx, void** gsum, long long* bytes_per_group, int* g_lo, int* g_hi)
{
    if (!ready(ctx)) return QR_EINVAL;
    if (gsum) *gsum = ctx->d_gsum;
    if (bytes_per_group) *bytes_per_group = (long long)sizeof(double2) * ctx->N * ctx->nGp;
    return qr_shard_plan(ctx->P.n_chunks, ctx->shard_rank, ctx->shard_world, nullptr, nullptr, g_lo, g_hi);
}

qr_status qr_picard_begin(qr_ctx* ctx)
{
    if (!ready(ctx)) return QR_EINVAL;
    if (ctx->cosine) return fail(ctx, QR_ENOTIMPL, "qr_picard_begin: the cosine basis is not supported");
    if (!ctx->d_gsum) return fail(ctx, QR_EINVAL, "qr_picard_begin: the context is not sharded (qr_shard, world > 1)");
    QR_CU(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned), ctx->stream));
    cudaError_t e = ctx->tree_slots ? launch_paths_tree(ctx->prec, ctx->gkind, ctx->gn, ctx->P, ctx->d_tree,
                                                        ctx->tree_stride, ctx->d_S, 0, ctx->N, ctx->d_counters,
                                                        ctx->d_status, ctx->stream)
                                    : launch_paths(ctx->prec, ctx->P, ctx->d_tab, ctx->d_first, ctx->d_packed,
                                                   ctx->row_stride, ctx->d_S, 0, ctx->N, ctx->d_counters,
                                                   ctx->d_status, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "path-and-series kernel");
    e = ctx->proj_nodes ? launch_project_tree(ctx->prec, ctx->gkind, ctx->gn, ctx->P, ctx->d_S, ctx->d_perm,
                                              ctx->d_partial, 0, ctx->N, ctx->stream)
                        : launch_project(ctx->prec, ctx->P, ctx->d_tab, ctx->d_first, ctx->d_S, ctx->d_partial, 0,
                                         ctx->N, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "projection kernel");
    int gl = 0, gh = 0;
    qr_shard_plan(ctx->P.n_chunks, ctx->shard_rank, ctx->shard_world, nullptr, nullptr, &gl, &gh);
    e = launch_group_sums(ctx->P, ctx->d_partial, ctx->d_gsum, gl, gh, 0, ctx->N, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "group sums");
    return QR_OK;
}

qr_status qr_picard_finish(qr_ctx* ctx, double* residual_out)
{
    if (!ready(ctx)) return QR_EINVAL;
    if (!ctx->d_gsum) return fail(ctx, QR_EINVAL, "qr_picard_finish: the context is not sharded (qr_shard, world > 1)");
    QR_CU(ctx, cudaMemsetAsync(ctx->d_counters + CNT_RESID, 0, sizeof(unsigned long long), ctx->stream));
    cudaError_t e = launch_reduce_groups(ctx->prec, ctx->P, ctx->d_gsum, ctx->d_alpha, ctx->nG, ctx->zero_idx,
                                         ctx->d_packed, ctx->row_stride, 0, ctx->N, ctx->d_counters, ctx->stream);
    if (e == cudaSuccess && ctx->tree_slots) e = pack_tree_rows(ctx, 0, ctx->N);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reduction kernel");
    ctx->stats.iterations++;
    const long long nonfinite_before = ctx->stats.nonfinite;
    qr_status s = check_device_status(ctx);
    if (s != QR_OK) return s;
    if (residual_out) {
        unsigned long long bits = ctx->h_counters[CNT_RESID];
        std::memcpy(residual_out, &bits, sizeof *residual_out);
    }
    if (ctx->stats.nonfinite > nonfinite_before) return fail(ctx, QR_ENONFINITE, "non-finite responses");
    return QR_OK;
}

qr_status qr_selftest_wait_timeout(qr_ctx* ctx)
{
    if (!ready(ctx)) return QR_EINVAL;
    QR_CU(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned), ctx->stream));
    QR_CU(ctx, launch_wait_selftest(ctx->d_status, ctx->stream));
    const qr_status s = check_device_status(ctx);
    QR_CU(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned), ctx->stream));
    QR_CU(ctx, cudaStreamSynchronize(ctx->stream));
    return s;
}

qr_status qr_backward_sweep(qr_ctx* ctx)
{
    if (!ready(ctx)) return QR_EINVAL;
    if (ctx->shard_world > 1) return fail(ctx, QR_EINVAL, "qr_backward_sweep: not for a sharded context");
    NvtxRange range("qr_backward_sweep");
    qr_status fs = take_iteration_fault(ctx);
    if (fs != QR_OK) return fs;
    QR_CU(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned), ctx->stream));
    for (int i = ctx->N - 1; i >= 0; --i) {
        qr_status s = run_rows(ctx, i, i + 1);
        if (s != QR_OK) return s;
    }
    ctx->stats.iterations++;
    const long long nonfinite_before = ctx->stats.nonfinite;
    qr_status s = check_device_status(ctx);
    if (s != QR_OK) return s;
    if (ctx->stats.nonfinite > nonfinite_before) return fail(ctx, QR_ENONFINITE, "non-finite responses");
    return QR_OK;
}

qr_status qr_eval(qr_ctx* ctx, int i, const double* x, long long n, double* y_out, int ptr_kind)
{
    if (!ready(ctx)) return QR_EINVAL;
    if (i < 0 || i > ctx->N || n < 0 || (n > 0 && (!x || !y_out)) || (ptr_kind != QR_HOST && ptr_kind != QR_DEVICE))
        return fail(ctx, QR_EINVAL, "qr_eval: bad arguments");
    if (n == 0) return QR_OK;
    const double* dx = x;
    double* dy = y_out;
    double* tmp = nullptr;
    if (ptr_kind == QR_HOST) {
        tmp = static_cast<double*>(ctx_malloc(ctx, sizeof(double) * (size_t)n * (ctx->d + 1)));
        if (!tmp) return fail(ctx, QR_ENOMEM, "qr_eval: device allocation failed");
        QR_CU(ctx, cudaMemcpyAsync(tmp, x, sizeof(double) * (size_t)n * ctx->d, cudaMemcpyHostToDevice, ctx->stream));
        dx = tmp;
        dy = tmp + (size_t)n * ctx->d;
    }
    const int use_g = (i == ctx->N && !ctx->trig_g) ? 1 : 0;
    const void* row = static_cast<const char*>(ctx->d_packed) + ctx->elem * (size_t)i * ctx->row_stride;
    cudaError_t e = ctx->cos_direct
                        ? launch_eval_cos(ctx->prec, ctx->P, ctx->d_cflags, ctx->cos_groups, row, dx, n, dy, use_g,
                                          ctx->stream)
                        : launch_eval(ctx->prec, ctx->P, ctx->d_tab, ctx->d_first, row, dx, n, dy, use_g, ctx->stream);
    if (e != cudaSuccess) {
        ctx_free(ctx, tmp);
        return cuda_fail(ctx, e, "evaluation kernel");
    }
    if (ptr_kind == QR_HOST) {
        QR_CU(ctx, cudaMemcpyAsync(y_out, dy, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream));
        QR_CU(ctx, cudaStreamSynchronize(ctx->stream));
        ctx_free(ctx, tmp);
    }
    QR_CU(ctx, cudaStreamSynchronize(ctx->stream));
    return QR_OK;
}

qr_status qr_gamma_size(const qr_ctx* ctx, int* n_gamma)
{
    if (!ready(ctx) || !n_gamma) return QR_EINVAL;
    *n_gamma = ctx->cosine ? ctx->nGn : ctx->nG;
    return QR_OK;
}

qr_status qr_gamma_list(const qr_ctx* ctx, int* k_out)
{
    if (!ready(ctx) || !k_out) return QR_EINVAL;
    const std::vector<int>& k = ctx->cosine ? ctx->kn : ctx->k;
    std::memcpy(k_out, k.data(), sizeof(int) * k.size());
    return QR_OK;
}

qr_status qr_get_coefs(const qr_ctx* ctx, double* alpha_out)
{
    if (!ready(ctx) || !alpha_out) return QR_EINVAL;
    qr_ctx* c = const_cast<qr_ctx*>(ctx);
    if (!ctx->cosine || ctx->cos_direct) {  // direct cosine rows hold (a_k, 0)
        QR_CU(c, cudaMemcpyAsync(alpha_out, ctx->d_alpha, sizeof(double2) * (size_t)ctx->N * ctx->nG,
                                 cudaMemcpyDeviceToHost, ctx->stream));
        QR_CU(c, cudaStreamSynchronize(ctx->stream));
        return QR_OK;
    }
    // cosine: a_k = c_k / zscale(k) from the unfolded rows
    std::vector<double2> z((size_t)ctx->N * ctx->nG);
    QR_CU(c, cudaMemcpyAsync(z.data(), ctx->d_alpha, sizeof(double2) * z.size(), cudaMemcpyDeviceToHost, ctx->stream));
    QR_CU(c, cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < ctx->N; ++i)
        for (int q = 0; q < ctx->nGn; ++q) {
            const int e = ctx->z_of_n[q];
            alpha_out[2 * ((size_t)i * ctx->nGn + q)] = z[(size_t)i * ctx->nG + e].x / ctx->zscale[e];
            alpha_out[2 * ((size_t)i * ctx->nGn + q) + 1] = 0.0;
        }
    return QR_OK;
}

qr_status qr_set_coefs(qr_ctx* ctx, const double* alpha_in)
{
    if (!ready(ctx) || !alpha_in) return QR_EINVAL;
    const int n_in = ctx->cosine ? ctx->nGn : ctx->nG;
    for (long long t = 0; t < 2ll * ctx->N * n_in; ++t)
        if (!std::isfinite(alpha_in[t])) return fail(ctx, QR_EINVAL, "qr_set_coefs: non-finite coefficient");
    std::vector<double2> z;
    const void* src = alpha_in;
    if (ctx->cos_direct) {
        z.resize((size_t)ctx->N * ctx->nG);
        for (size_t t = 0; t < z.size(); ++t) z[t] = make_double2(alpha_in[2 * t], 0.0);
        src = z.data();
    } else if (ctx->cosine) {
        // unfold the cosine coefficients (real parts) onto the Z^d set
        z.resize((size_t)ctx->N * ctx->nG);
        for (int i = 0; i < ctx->N; ++i)
            for (int e = 0; e < ctx->nG; ++e)
                z[(size_t)i * ctx->nG + e] =
                    make_double2(alpha_in[2 * ((size_t)i * ctx->nGn + ctx->n_of_z[e])] * ctx->zscale[e], 0.0);
        src = z.data();
    }
    QR_CU(ctx, cudaMemcpyAsync(ctx->d_alpha, src, sizeof(double2) * (size_t)ctx->N * ctx->nG,
                               cudaMemcpyHostToDevice, ctx->stream));
    qr_status s = repack_all(ctx);
    if (s != QR_OK) return s;
    QR_CU(ctx, cudaStreamSynchronize(ctx->stream));
    return QR_OK;
}

qr_status qr_get_responses(const qr_ctx* ctx, int i, double* S_out)
{
    if (!ready(ctx) || !S_out || i < 0 || i >= ctx->N) return QR_EINVAL;
    qr_ctx* c = const_cast<qr_ctx*>(ctx);
    const size_t M = (size_t)ctx->P.M;
    if (ctx->prec == QR_FP64) {
        QR_CU(c, cudaMemcpyAsync(S_out, static_cast<double*>(ctx->d_S) + (size_t)i * M, sizeof(double) * M,
                                 cudaMemcpyDeviceToHost, ctx->stream));
        QR_CU(c, cudaStreamSynchronize(ctx->stream));
    } else {
        std::vector<float> tmp(M);
        QR_CU(c, cudaMemcpyAsync(tmp.data(), static_cast<float*>(ctx->d_S) + (size_t)i * M, sizeof(float) * M,
                                 cudaMemcpyDeviceToHost, ctx->stream));
        QR_CU(c, cudaStreamSynchronize(ctx->stream));
        for (size_t t = 0; t < M; ++t) S_out[t] = tmp[t];
    }
    return QR_OK;
}

qr_status qr_set_profiling(qr_ctx* ctx, int on)
{
    if (!ready(ctx)) return QR_EINVAL;
    ctx->profiling = on != 0;
    return QR_OK;
}

qr_status qr_get_stats(const qr_ctx* ctx, qr_stats_t* out)
{
    if (!ready(ctx) || !out) return QR_EINVAL;
    *out = ctx->stats;
    return QR_OK;
}

qr_status qr_test_points(const qr_ctx* ctx, int i, long long n, double* x_out)
{
    if (!ready(ctx) || !x_out || n < 0 || i < 0 || i > ctx->N) return QR_EINVAL;
    if (n == 0) return QR_OK;
    qr_ctx* c = const_cast<qr_ctx*>(ctx);
    double* d = static_cast<double*>(ctx_malloc(c, sizeof(double) * (size_t)n * ctx->d));
    if (!d) return fail(c, QR_ENOMEM, "qr_test_points: device allocation failed");
    cudaError_t e = launch_test_points(ctx->P, i, n, d, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(x_out, d, sizeof(double) * (size_t)n * ctx->d, cudaMemcpyDeviceToHost, ctx->stream);
    ctx_free(c, d);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "test points");
    return QR_OK;
}

qr_status qr_tree_layout(int kind, int d, int n, int* n_slots, int* n_terms, int* idx, double* coef)
{
    if ((kind != QR_G_LINF && kind != QR_G_L1) || d < 1 || d > kDMaxFourier || n < 1 || n > 31 || !n_slots)
        return QR_EINVAL;
    std::vector<int> K;
    enumerate_gamma(kind, d, n, K);
    std::vector<TreeMap> map;
    if (!build_tree_map(kind, d, n, K, map)) return QR_EINVAL;
    *n_slots = (int)map.size();
    if (n_terms) *n_terms = kTreeTerms;
    for (size_t s = 0; s < map.size(); ++s)
        for (int h = 0; h < 2; ++h)
            for (int t = 0; t < kTreeTerms; ++t) {
                const size_t o = (s * 2 + h) * kTreeTerms + t;
                if (idx) idx[o] = map[s].c[h][t] != 0.0 ? map[s].i[h][t] : -1;
                if (coef) coef[o] = map[s].c[h][t];
            }
    return QR_OK;
}

qr_status qr_philox_words(const uint32_t* ctr_key, long long n, uint32_t* out)
{
    if (n < 0 || (n > 0 && (!ctr_key || !out))) return QR_EINVAL;
    if (n == 0) return QR_OK;
    uint32_t *d_in = nullptr, *d_out = nullptr;
    if (cudaMalloc(&d_in, sizeof(uint32_t) * 6 * (size_t)n) != cudaSuccess) return QR_ENOMEM;
    if (cudaMalloc(&d_out, sizeof(uint32_t) * 4 * (size_t)n) != cudaSuccess) {
        cudaFree(d_in);
        return QR_ENOMEM;
    }
    qr_status s = QR_OK;
    if (cudaMemcpy(d_in, ctr_key, sizeof(uint32_t) * 6 * (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess ||
        launch_philox(d_in, n, d_out, 0) != cudaSuccess ||
        cudaMemcpy(out, d_out, sizeof(uint32_t) * 4 * (size_t)n, cudaMemcpyDeviceToHost) != cudaSuccess)
        s = QR_ECUDA;
    cudaFree(d_in);
    cudaFree(d_out);
    return s;
}

qr_status qr_sample(int d, const qr_nu* nu, unsigned long long seed, int instance, int i, long long m0, long long n,
                    int j, int precision, double* u_out, double* x_out, double* z_out)
{
    if (d < 1 || d > kDMaxFourier || !nu || n < 0 || m0 < 0 || i < 0 || i >= 65536 || instance < 0 || instance >= 4096 ||
        (precision != QR_FP32 && precision != QR_FP64))
        return QR_EINVAL;
    if (n == 0) return QR_OK;
    QrParams P{};
    P.d = d;
    P.nu_kind = nu->kind;
    P.mu = nu->kind == QR_NU_LOMAX ? nu->mu : (nu->kind == QR_NU_STUDENT2 ? 2.0 : 1.0);
    P.inv_mu = 1.0 / P.mu;
    P.mu_is3 = nu->kind == QR_NU_LOMAX && nu->mu == 3.0;
    P.key0 = (uint32_t)(seed & 0xffffffffull);
    P.key1 = (uint32_t)(seed >> 32);
    P.instance = instance;
    double* buf = nullptr;
    const size_t each = (size_t)n * d;
    if (cudaMalloc(&buf, sizeof(double) * 3 * each) != cudaSuccess) return QR_ENOMEM;
    qr_status s = QR_OK;
    if (launch_sample(precision, P, i, m0, n, j, buf, buf + each, buf + 2 * each, 0) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess)
        s = QR_ECUDA;
    if (s == QR_OK && u_out && cudaMemcpy(u_out, buf, sizeof(double) * each, cudaMemcpyDeviceToHost) != cudaSuccess)
        s = QR_ECUDA;
    if (s == QR_OK && x_out &&
        cudaMemcpy(x_out, buf + each, sizeof(double) * each, cudaMemcpyDeviceToHost) != cudaSuccess)
        s = QR_ECUDA;
    if (s == QR_OK && z_out &&
        cudaMemcpy(z_out, buf + 2 * each, sizeof(double) * each, cudaMemcpyDeviceToHost) != cudaSuccess)
        s = QR_ECUDA;
    cudaFree(buf);
    return s;
}

qr_status qr_sample_normals_tree(int d, unsigned long long seed, int instance, int i, long long m0, long long n,
                                 int j, double* z_out)
{
    if (d < 1 || d > kDMaxFourier || !z_out || n < 0 || m0 < 0 || i < 0 || i >= 65536 || instance < 0 || instance >= 4096)
        return QR_EINVAL;
    if (n == 0) return QR_OK;
    QrParams P{};
    P.d = d;
    P.key0 = (uint32_t)(seed & 0xffffffffull);
    P.key1 = (uint32_t)(seed >> 32);
    P.instance = instance;
    double* buf = nullptr;
    const size_t bytes = sizeof(double) * (size_t)n * d;
    if (cudaMalloc(&buf, bytes) != cudaSuccess) return QR_ENOMEM;
    qr_status s = QR_OK;
    if (launch_normals_tree(P, i, m0, n, j, buf, 0) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(z_out, buf, bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
        s = QR_ECUDA;
    cudaFree(buf);
    return s;
}

}  // extern "C"

// ------------------------------------------------------------------ batches
// instances that share their sample points, run by the tensor-core kernel
struct BatchGroup {
    int kind = 0, d = 0, n = 0;
    std::vector<int> members;
    QrParams P{};
    GroupInst* d_inst = nullptr;
    void* d_apack = nullptr;
    const int* d_perm = nullptr;
    int nG = 0, zero_idx = 0;
    unsigned* status = nullptr;
};

struct qr_batch {
    std::vector<qr_ctx*> ctx;
    std::vector<BatchGroup> groups;
    std::vector<char> grouped;  // per instance
    int group_min = 16;
    cudaStream_t stream = nullptr;
    BatchInst* d_inst = nullptr;
    BatchItem* d_items = nullptr;
    unsigned* d_next = nullptr;
    int n_items = 0;
    size_t max_rowbytes = 0;
    int grid = 0, tiles_per_item = 1;
    bool tuned = false;
    cudaGraphExec_t graph = nullptr;
    cudaEvent_t ev[2] = {};
    double tune_ms[8] = {};
    std::string err;
    // one finishing launch (projection, reduction, repacks) for all instances
    // when every instance has a compiled tiled projection
    bool fused = false;
    FinishInst* d_fin = nullptr;
    FinishGroup* d_fgroups = nullptr;
    int4* d_fitems = nullptr;
    long long n_fitems = 0;
    unsigned* d_row_done = nullptr;
    unsigned* d_grp_done = nullptr;
    unsigned long long* d_resid = nullptr;
};

namespace {

qr_status bfail(qr_batch* b, qr_status s, const std::string& m)
{
    if (b) b->err = m;
    return s;
}

// device tables of a batch: through its first context's allocator
bool balloc(qr_batch* b, void** p, size_t bytes)
{
    *p = ctx_malloc(b->ctx[0], bytes);
    // filled by synchronous copies: no earlier work on the stream may still use it
    return *p != nullptr && cudaStreamSynchronize(b->ctx[0]->stream) == cudaSuccess;
}
void bfree(qr_batch* b, void* p)
{
    if (p && !b->ctx.empty()) {
        cudaStreamSynchronize(b->ctx[0]->stream);
        ctx_free(b->ctx[0], p);
    }
}

// items of all instances, `tpi` tiles per item
std::vector<BatchItem> batch_items(const qr_batch* b, int tpi)
{
    const int tp = batch_tile_paths();
    std::vector<BatchItem> items;
    for (int q = 0; q < (int)b->ctx.size(); ++q) {
        if (b->grouped[q]) continue;
        const qr_ctx* c = b->ctx[q];
        const int tiles = (int)((c->P.M + tp - 1) / tp);
        for (int i = 0; i < c->N; ++i)
            for (int t = 0; t < tiles; t += tpi) items.push_back(BatchItem{q, i, t, std::min(tpi, tiles - t)});
    }
    // class by class (the class with the most work first), longest rows
    // first within a class: the CTAs running at any time mostly execute the
    // same compiled body and share the instruction caches (8 % faster on the
    // 256-instance workload than one longest-first order across classes)
    std::vector<double> work(64, 0.0);
    auto cls = [&](const BatchItem& x) {
        const qr_ctx* c = b->ctx[x.inst];
        return batch_class(c->gkind, c->d, c->gn);
    };
    for (const BatchItem& x : items)
        work[cls(x)] += (double)(b->ctx[x.inst]->N - x.i) * x.ntiles * (b->ctx[x.inst]->tree_slots);
    std::stable_sort(items.begin(), items.end(), [&](const BatchItem& x, const BatchItem& y) {
        const int cx = cls(x), cy = cls(y);
        if (cx != cy) return work[cx] > work[cy] || (work[cx] == work[cy] && cx < cy);
        return b->ctx[x.inst]->N - x.i > b->ctx[y.inst]->N - y.i;
    });
    return items;
}

qr_status batch_set_items(qr_batch* b, int tpi)
{
    std::vector<BatchItem> items = batch_items(b, tpi);
    bfree(b, b->d_items);
    b->d_items = nullptr;
    if (!balloc(b, reinterpret_cast<void**>(&b->d_items), sizeof(BatchItem) * std::max<size_t>(1, items.size())))
        return bfail(b, QR_ENOMEM, "batch items");
    if (cudaMemcpy(b->d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return bfail(b, QR_ECUDA, "copy batch items");
    b->n_items = (int)items.size();
    b->tiles_per_item = tpi;
    return QR_OK;
}

qr_status batch_paths(qr_batch* b)
{
    cudaError_t e = cudaMemsetAsync(b->d_next, 0, sizeof(unsigned), b->stream);
    if (e == cudaSuccess)
        e = launch_paths_batch(b->d_inst, b->d_items, b->n_items, b->d_next, b->max_rowbytes, b->grid, b->stream);
    for (const BatchGroup& g : b->groups) {
        // the fused path repacks the group blocks in its finishing kernel
        if (e == cudaSuccess && !b->fused)
            e = launch_pack_group(g.kind, g.d, g.n, g.d_inst, (int)g.members.size(), g.nG, g.zero_idx, g.d_perm,
                                  g.d_apack, g.P.N, b->stream);
        if (e == cudaSuccess)
            e = launch_paths_group(g.kind, g.d, g.n, g.P, g.d_inst, (int)g.members.size(), g.d_apack, g.status,
                                   b->stream);
    }
    return e == cudaSuccess ? QR_OK : bfail(b, QR_ECUDA, std::string("batch path kernel: ") + cudaGetErrorString(e));
}

// same Euler paths and the same basis: every input of the path simulation
// and of the index set agrees; the driver and g are the cubic/cosine pair
bool shares_points(const qr_ctx* a, const qr_ctx* c)
{
    const QrParams &p = a->P, &q = c->P;
    if (a->d != c->d || a->N != c->N || p.M != q.M || a->gkind != c->gkind || a->gn != c->gn) return false;
    if (p.nu_kind != q.nu_kind || p.mu != q.mu || p.T != q.T || p.sig_diag != q.sig_diag) return false;
    if (p.key0 != q.key0 || p.key1 != q.key1 || p.instance != q.instance || p.lattice_n != q.lattice_n) return false;
    for (int l = 0; l < a->d; ++l)
        if (p.b[l] != q.b[l]) return false;
    for (int t = 0; t < kDMax * kDMax; ++t)
        if (p.sig[t] != q.sig[t]) return false;
    return true;
}

void free_groups(qr_batch* b)
{
    for (BatchGroup& g : b->groups) {
        bfree(b, g.d_inst);
        bfree(b, g.d_apack);
    }
    b->groups.clear();
    b->grouped.assign(b->ctx.size(), 0);
}

// sets of at least group_min instances sharing their points (and with a
// compiled shared-point kernel) go to the tensor-core path
qr_status batch_build_groups(qr_batch* b)
{
    free_groups(b);
    const int n = (int)b->ctx.size();
    std::vector<char> seen(n, 0);
    for (int q = 0; q < n && b->group_min > 0; ++q) {
        if (seen[q]) continue;
        const qr_ctx* c = b->ctx[q];
        if (!group_supported(c->gkind, c->d, c->gn) || !c->d_perm || c->N > kGroupNMax) continue;
        if (c->P.f_kind != QR_F_CUBIC_MANUF || c->P.g_kind != QR_GT_COS || c->P.q_damp != 0.0) continue;
        std::vector<int> mem;
        for (int r = q; r < n; ++r) {
            const qr_ctx* e = b->ctx[r];
            if (!seen[r] && e->P.f_kind == QR_F_CUBIC_MANUF && e->P.g_kind == QR_GT_COS && e->P.q_damp == 0.0 &&
                shares_points(c, e))
                mem.push_back(r);
        }
        if ((int)mem.size() < b->group_min) continue;
        BatchGroup g;
        g.kind = c->gkind;
        g.d = c->d;
        g.n = c->gn;
        g.members = mem;
        g.P = c->P;
        g.d_perm = c->d_perm;
        g.nG = c->nG;
        g.zero_idx = c->zero_idx;
        g.status = c->d_status;
        std::vector<GroupInst> gi(mem.size());
        for (size_t t = 0; t < mem.size(); ++t) {
            const qr_ctx* e = b->ctx[mem[t]];
            seen[mem[t]] = 1;
            GroupInst& I = gi[t];
            std::memset(&I, 0, sizeof I);
            for (int l = 0; l < e->d; ++l) {
                I.p.fs[l] = (float)e->P.f_s[l];
                I.p.gs[l] = (float)e->P.g_s[l];
            }
            I.p.f_c = (float)e->P.f_c;
            I.p.clamp_L = (float)e->P.clamp_L;
            for (int j = 0; j < e->N; ++j) I.fexp[j] = (float)e->P.fexp[j];
            I.S = e->d_S;
            I.alpha = e->d_alpha;
        }
        const int ntg = ((int)mem.size() + 31) / 32;
        const size_t abytes = (size_t)c->N * ntg * 2 * (size_t)group_block_elems(g.kind, g.d, g.n) * 2;
        const bool ok = balloc(b, reinterpret_cast<void**>(&g.d_inst), sizeof(GroupInst) * gi.size()) &&
                        balloc(b, &g.d_apack, abytes);
        b->groups.push_back(g);
        if (!ok) return bfail(b, QR_ENOMEM, "batch group allocation");
        if (cudaMemcpy(g.d_inst, gi.data(), sizeof(GroupInst) * gi.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return bfail(b, QR_ECUDA, "copy group instances");
        for (int r : mem) b->grouped[r] = 1;
    }
    return QR_OK;
}

void free_finish(qr_batch* b)
{
    void* ptrs[] = {b->d_fin, b->d_fgroups, b->d_fitems, b->d_row_done, b->d_grp_done, b->d_resid};
    for (void* p : ptrs) bfree(b, p);
    b->d_fin = nullptr;
    b->d_fgroups = nullptr;
    b->d_fitems = nullptr;
    b->d_row_done = nullptr;
    b->d_grp_done = nullptr;
    b->d_resid = nullptr;
    b->n_fitems = 0;
    b->fused = false;
}

// the finishing kernel's instance and group tables, its work items (class
// by class, then instance, row, chunk) and zeroed arrival counters
qr_status batch_build_finish(qr_batch* b)
{
    free_finish(b);
    const int n = (int)b->ctx.size();
    for (const qr_ctx* c : b->ctx)
        if (!c->proj_nodes || !c->d_perm || c->shard_world != 1) return QR_OK;  // per-instance path
    std::vector<int> grp_of(n, -1);
    std::vector<FinishGroup> fg;
    int grows = 0;
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        const BatchGroup& g = b->groups[gi];
        const int gcls = finish_group_class(g.kind, g.d, g.n);
        if (gcls < 0) return QR_OK;
        for (int q : g.members) grp_of[q] = (int)gi;
        FinishGroup G{};
        G.gcls = gcls;
        G.inst = g.d_inst;
        G.n_inst = (int)g.members.size();
        G.nG = g.nG;
        G.zero_idx = g.zero_idx;
        G.perm = g.d_perm;
        G.Bpack = static_cast<uint8_t*>(g.d_apack);
        G.row_base = grows;
        grows += g.P.N;
        fg.push_back(G);
    }
    std::vector<FinishInst> fi(n);
    int rows = 0;
    for (int q = 0; q < n; ++q) {
        const qr_ctx* c = b->ctx[q];
        FinishInst& F = fi[q];
        std::memset(&F, 0, sizeof F);
        F.P = c->P;
        F.cls = batch_class(c->gkind, c->d, c->gn);
        F.S = static_cast<const float*>(c->d_S);
        F.partial = c->d_partial;
        F.alpha = c->d_alpha;
        F.packed = static_cast<float2*>(c->d_packed);
        F.row_stride = c->row_stride;
        F.tree = static_cast<float2*>(c->d_tree);
        F.tree_stride = c->tree_stride;
        F.tmap = c->d_tmap;
        F.tree_slots = c->tree_slots;
        F.perm = c->d_perm;
        F.nG = c->nG;
        F.zero_idx = c->zero_idx;
        F.row_base = rows;
        F.group = grp_of[q];
        rows += c->N;
    }
    std::vector<int4> items;
    for (int cls = 0; cls < 64; ++cls)
        for (int q = 0; q < n; ++q) {
            if (fi[q].cls != cls) continue;
            for (int i = 0; i < b->ctx[q]->N; ++i)
                for (int ch = 0; ch < fi[q].P.n_chunks; ++ch) items.push_back(make_int4(q, i, ch, 0));
        }
    const bool ok =
        balloc(b, reinterpret_cast<void**>(&b->d_fin), sizeof(FinishInst) * n) &&
        balloc(b, reinterpret_cast<void**>(&b->d_fgroups), sizeof(FinishGroup) * std::max<size_t>(1, fg.size())) &&
        balloc(b, reinterpret_cast<void**>(&b->d_fitems), sizeof(int4) * std::max<size_t>(1, items.size())) &&
        balloc(b, reinterpret_cast<void**>(&b->d_row_done), sizeof(unsigned) * std::max(1, rows)) &&
        balloc(b, reinterpret_cast<void**>(&b->d_grp_done), sizeof(unsigned) * std::max(1, grows)) &&
        balloc(b, reinterpret_cast<void**>(&b->d_resid), sizeof(unsigned long long) * n);
    if (!ok) {
        free_finish(b);
        return bfail(b, QR_ENOMEM, "batch finishing tables");
    }
    if (cudaMemcpy(b->d_fin, fi.data(), sizeof(FinishInst) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        (!fg.empty() && cudaMemcpy(b->d_fgroups, fg.data(), sizeof(FinishGroup) * fg.size(), cudaMemcpyHostToDevice) !=
                            cudaSuccess) ||
        cudaMemcpy(b->d_fitems, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->d_row_done, 0, sizeof(unsigned) * std::max(1, rows)) != cudaSuccess ||
        cudaMemset(b->d_grp_done, 0, sizeof(unsigned) * std::max(1, grows)) != cudaSuccess) {
        free_finish(b);
        return bfail(b, QR_ECUDA, "copy batch finishing tables");
    }
    b->n_fitems = (long long)items.size();
    b->fused = true;
    return QR_OK;
}

// projection, reduction and repacks of every instance in one launch
qr_status batch_rest_fused(qr_batch* b)
{
    cudaError_t e = cudaMemsetAsync(b->d_resid, 0, sizeof(unsigned long long) * b->ctx.size(), b->stream);
    if (e == cudaSuccess)
        e = launch_finish_batch(b->d_fin, b->d_fitems, b->n_fitems, b->d_fgroups, b->d_row_done, b->d_grp_done,
                                b->d_resid, b->stream);
    return e == cudaSuccess ? QR_OK : bfail(b, QR_ECUDA, std::string("batch finishing kernel: ") + cudaGetErrorString(e));
}

// projection, reduction and repack of every instance (single-instance kernels)
qr_status batch_rest(qr_batch* b)
{
    if (b->fused) return batch_rest_fused(b);
    for (qr_ctx* c : b->ctx) {
        cudaError_t e = cudaMemsetAsync(c->d_counters + CNT_RESID, 0, sizeof(unsigned long long), b->stream);
        if (e == cudaSuccess)
            e = c->proj_nodes ? launch_project_tree(c->prec, c->gkind, c->gn, c->P, c->d_S, c->d_perm, c->d_partial,
                                                    0, c->N, b->stream)
                              : launch_project(c->prec, c->P, c->d_tab, c->d_first, c->d_S, c->d_partial, 0, c->N,
                                               b->stream);
        if (e == cudaSuccess)
            e = launch_reduce(c->prec, c->P, c->d_partial, c->d_alpha, c->nG, c->zero_idx, c->d_packed,
                              c->row_stride, 0, c->N, c->d_counters, b->stream);
        if (e == cudaSuccess)
            e = launch_pack_tree(c->prec, c->d_alpha, c->nG, c->d_tmap, c->tree_slots, c->d_tree, c->tree_stride,
                                 c->N, b->stream);
        if (e != cudaSuccess) return bfail(b, QR_ECUDA, std::string("batch projection: ") + cudaGetErrorString(e));
    }
    return QR_OK;
}

}  // namespace

extern "C" {

qr_status qr_batch_create(qr_batch** out, qr_ctx* const* ctxs, int n)
{
    if (!out || !ctxs || n < 1) return QR_EINVAL;
    *out = nullptr;
    qr_batch* b = new (std::nothrow) qr_batch();
    if (!b) return QR_ENOMEM;
    *out = b;
    size_t maxrow = 16;
    std::vector<BatchInst> inst(n);
    for (int q = 0; q < n; ++q) {
        qr_ctx* c = ctxs[q];
        if (!ready(c)) return bfail(b, QR_EINVAL, "batch: instance " + std::to_string(q) + " is not a context");
        if (c->prec != QR_FP32) return bfail(b, QR_EINVAL, "batch: instances must use QR_FP32");
        if (c->cosine) return bfail(b, QR_ENOTIMPL, "batch: the cosine basis is not supported");
        if (c->shard_world > 1) return bfail(b, QR_EINVAL, "batch: instances must not be sharded");
        const int cls = batch_class(c->gkind, c->d, c->gn);
        if (cls < 0 || !c->tree_slots)
            return bfail(b, QR_ENOTIMPL, "batch: index set of instance " + std::to_string(q) + " has no compiled class");
        if (q > 0 && c->stream != ctxs[0]->stream) return bfail(b, QR_EINVAL, "batch: instances must share a stream");
        b->ctx.push_back(c);
        inst[q].P = c->P;
        inst[q].cls = cls;
        inst[q].tree = c->d_tree;
        inst[q].tree_stride = c->tree_stride;
        inst[q].S = c->d_S;
        inst[q].counters = c->d_counters;
        inst[q].status = c->d_status;
        maxrow = std::max(maxrow, (size_t)c->tree_stride * sizeof(float2));
    }
    b->stream = ctxs[0]->stream;
    b->max_rowbytes = (maxrow + 15) & ~size_t(15);
    if (!balloc(b, reinterpret_cast<void**>(&b->d_inst), sizeof(BatchInst) * n) ||
        !balloc(b, reinterpret_cast<void**>(&b->d_next), sizeof(unsigned)))
        return bfail(b, QR_ENOMEM, "batch allocation");
    if (cudaMemcpy(b->d_inst, inst.data(), sizeof(BatchInst) * n, cudaMemcpyHostToDevice) != cudaSuccess)
        return bfail(b, QR_ECUDA, "copy batch instances");
    for (auto& e : b->ev)
        if (cudaEventCreate(&e) != cudaSuccess) return bfail(b, QR_ECUDA, "events");
    const int per_sm = batch_blocks_per_sm(b->max_rowbytes);
    if (per_sm < 1) return bfail(b, QR_ENOTIMPL, "batch: rows too large for shared memory");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    b->grid = per_sm * sms;
    qr_status gs = batch_build_groups(b);
    if (gs == QR_OK) gs = batch_build_finish(b);
    if (gs != QR_OK) return gs;
    return batch_set_items(b, 4);
}

qr_status qr_batch_set_grouping(qr_batch* b, int min_group)
{
    if (!b || b->ctx.empty() || min_group < 0) return QR_EINVAL;
    if (b->tuned) return bfail(b, QR_EINVAL, "batch: grouping is fixed after the first iteration");
    b->group_min = min_group;
    qr_status s = batch_build_groups(b);
    if (s == QR_OK) s = batch_build_finish(b);
    return s == QR_OK ? batch_set_items(b, b->tiles_per_item) : s;
}

qr_status qr_batch_groups(const qr_batch* b, int* n_groups, int* n_grouped)
{
    if (!b) return QR_EINVAL;
    int k = 0;
    for (const BatchGroup& g : b->groups) k += (int)g.members.size();
    if (n_groups) *n_groups = (int)b->groups.size();
    if (n_grouped) *n_grouped = k;
    return QR_OK;
}

qr_status qr_batch_picard_step(qr_batch* b, int n_iter, double* max_residual)
{
    if (!b || b->ctx.empty() || !b->d_inst || n_iter < 0) return QR_EINVAL;
    for (qr_ctx* c : b->ctx)
        if (cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), b->stream) != cudaSuccess)
            return bfail(b, QR_ECUDA, "reset status");
    // the fused path repacks group blocks from the finished rows; coefficients
    // set from the host since then (or never packed) are packed here
    if (b->fused)
        for (const BatchGroup& g : b->groups) {
            bool changed = false;
            for (int q : g.members) changed = changed || b->ctx[q]->coefs_changed;
            if (!changed) continue;
            if (launch_pack_group(g.kind, g.d, g.n, g.d_inst, (int)g.members.size(), g.nG, g.zero_idx, g.d_perm,
                                  g.d_apack, g.P.N, b->stream) != cudaSuccess)
                return bfail(b, QR_ECUDA, "group coefficient blocks");
            for (int q : g.members) b->ctx[q]->coefs_changed = false;
        }
    if (!b->tuned && n_iter > 0) {
        // autotuner: time the persistent kernel for a few item sizes and
        // grids on the first iteration (it only rewrites the responses)
        const int tpis[] = {1, 4, 16};
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int per_sm = batch_blocks_per_sm(b->max_rowbytes);
        const int grids[] = {per_sm * sms, std::max(1, per_sm - 1) * sms};
        float best = 1e30f;
        int best_t = 4, best_g = b->grid, k = 0;
        for (int tpi : tpis)
            for (int g : grids) {
                qr_status s = batch_set_items(b, tpi);
                if (s != QR_OK) return s;
                b->grid = g;
                cudaEventRecord(b->ev[0], b->stream);
                s = batch_paths(b);
                if (s != QR_OK) return s;
                cudaEventRecord(b->ev[1], b->stream);
                float ms = 0.f;
                if (cudaEventSynchronize(b->ev[1]) != cudaSuccess ||
                    cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]) != cudaSuccess)
                    return bfail(b, QR_ECUDA, "autotune timing");
                if (k < 8) b->tune_ms[k++] = ms;
                if (ms < best) best = ms, best_t = tpi, best_g = g;
            }
        qr_status s = batch_set_items(b, best_t);
        if (s != QR_OK) return s;
        b->grid = best_g;
        for (qr_ctx* c : b->ctx)
            cudaMemsetAsync(c->d_counters, 0, sizeof(unsigned long long) * CNT_N, b->stream);
        b->tuned = true;
        // capture one iteration
        cudaGraph_t g = nullptr;
        bool ok = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            qr_status s1 = batch_paths(b), s2 = s1 == QR_OK ? batch_rest(b) : s1;
            ok = cudaStreamEndCapture(b->stream, &g) == cudaSuccess && s2 == QR_OK && g &&
                 cudaGraphInstantiate(&b->graph, g, 0) == cudaSuccess;
            if (g) cudaGraphDestroy(g);
        }
        if (!ok) {
            cudaGetLastError();
            b->graph = nullptr;
            b->err.clear();
        }
    }
    for (int q = 0; q < n_iter; ++q) {
        if (b->graph) {
            if (cudaGraphLaunch(b->graph, b->stream) != cudaSuccess) return bfail(b, QR_ECUDA, "graph launch");
        } else {
            qr_status s = batch_paths(b);
            if (s == QR_OK) s = batch_rest(b);
            if (s != QR_OK) return s;
        }
    }
    double rmax = 0.0;
    qr_status worst = QR_OK;
    for (qr_ctx* c : b->ctx) {
        if (n_iter > 0) c->stats.iterations += n_iter;
        const long long before = c->stats.nonfinite;
        qr_status s = check_device_status(c);
        if (s != QR_OK) {
            b->err = c->err;
            worst = s;
            continue;
        }
        if (c->stats.nonfinite > before) worst = QR_ENONFINITE;
        if (!b->fused) {
            double r;
            std::memcpy(&r, &c->h_counters[CNT_RESID], sizeof r);
            rmax = std::max(rmax, r);
        }
    }
    if (b->fused && n_iter > 0) {
        std::vector<unsigned long long> h(b->ctx.size());
        if (cudaMemcpy(h.data(), b->d_resid, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost) !=
            cudaSuccess)
            return bfail(b, QR_ECUDA, "read residuals");
        for (unsigned long long bits : h) {
            double r;
            std::memcpy(&r, &bits, sizeof r);
            rmax = std::max(rmax, r);
        }
    }
    if (max_residual) *max_residual = n_iter > 0 ? rmax : 0.0;
    return worst;
}

qr_status qr_batch_info(const qr_batch* b, int* tiles_per_item, int* grid, double* tune_ms /* 6 values */)
{
    if (!b) return QR_EINVAL;
    if (tiles_per_item) *tiles_per_item = b->tiles_per_item;
    if (grid) *grid = b->grid;
    if (tune_ms)
        for (int k = 0; k < 6; ++k) tune_ms[k] = b->tune_ms[k];
    return QR_OK;
}

const char* qr_batch_last_error(const qr_batch* b) { return b ? b->err.c_str() : "no batch"; }

void qr_batch_destroy(qr_batch* b)
{
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    bfree(b, b->d_inst);
    bfree(b, b->d_items);
    bfree(b, b->d_next);
    free_finish(b);
    free_groups(b);
    for (auto& e : b->ev)
        if (e) cudaEventDestroy(e);
    delete b;
}

}  // extern "C"
