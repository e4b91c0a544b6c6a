// qr_fast_paper.cu -- path-and-series tree kernels for the index sets of
// the paper's own experiments (Sec. 5), in their unfolded Z^d form: the
// one-dimensional Gamma_F(K) with K = 100, 150, 200 (|k| <= K) and the
// two-dimensional total-degree sets Gamma_T(20, 25, 31) (|k|_1 <= n).
// Compiled apart to keep build times parallel. The two-dimensional classes
// need more than 128 registers: 3 resident CTAs per SM here.
#define QR_TREE_MINB 3
#include "qr_tree.cuh"

namespace qr {

#define QR_TREE_PAPER(X) \
    X(QR_G_LINF, 1, 100) \
    X(QR_G_LINF, 1, 150) \
    X(QR_G_LINF, 1, 200) \
    X(QR_G_L1, 2, 20)    \
    X(QR_G_L1, 2, 25)    \
    X(QR_G_L1, 2, 31)

int tree_slots_paper(int kind, int d, int n)
{
#define QR_X(K, DD, NNN) \
    if (kind == K && d == DD && n == NNN) return tree_slots_t<DD, NNN, K>();
    QR_TREE_PAPER(QR_X)
#undef QR_X
    return 0;
}

cudaError_t launch_paths_tree_paper(int prec, int kind, int n, const QrParams& P, const void* tree,
                                    long long row_stride, void* S, int i_lo, int i_hi, unsigned long long* counters,
                                    unsigned* status, cudaStream_t st)
{
#define QR_X(K, DD, NNN)                                                                                      \
    if (kind == K && P.d == DD && n == NNN)                                                                   \
        return prec == QR_FP32                                                                                \
                   ? paths_tree_t<float, DD, NNN, K>(P, tree, row_stride, S, i_lo, i_hi, counters, status, st) \
                   : paths_tree_t<double, DD, NNN, K>(P, tree, row_stride, S, i_lo, i_hi, counters, status, st);
    QR_TREE_PAPER(QR_X)
#undef QR_X
    return cudaErrorInvalidValue;
}

}  // namespace qr
