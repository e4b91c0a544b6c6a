// qr_fast_more.cu -- path-and-series tree kernels for the further index
// sets of the multi-instance engine (compiled apart to keep build times
// parallel).
#include "qr_tree.cuh"

namespace qr {

#define QR_TREE_MORE(X) \
    X(QR_G_L1, 3, 5)    \
    X(QR_G_L1, 5, 4)    \
    X(QR_G_L1, 6, 3)    \
    X(QR_G_L1, 6, 4)    \
    X(QR_G_L1, 7, 3)    \
    X(QR_G_L1, 8, 3)

int tree_slots_more(int kind, int d, int n)
{
#define QR_X(K, DD, NNN) \
    if (kind == K && d == DD && n == NNN) return tree_slots_t<DD, NNN, K>();
    QR_TREE_MORE(QR_X)
#undef QR_X
    return tree_slots_paper(kind, d, n);
}

cudaError_t launch_paths_tree_more(int prec, int kind, int n, const QrParams& P, const void* tree,
                                   long long row_stride, void* S, int i_lo, int i_hi, unsigned long long* counters,
                                   unsigned* status, cudaStream_t st)
{
#define QR_X(K, DD, NNN)                                                                                      \
    if (kind == K && P.d == DD && n == NNN)                                                                   \
        return prec == QR_FP32                                                                                \
                   ? paths_tree_t<float, DD, NNN, K>(P, tree, row_stride, S, i_lo, i_hi, counters, status, st) \
                   : paths_tree_t<double, DD, NNN, K>(P, tree, row_stride, S, i_lo, i_hi, counters, status, st);
    QR_TREE_MORE(QR_X)
#undef QR_X
    return launch_paths_tree_paper(prec, kind, n, P, tree, row_stride, S, i_lo, i_hi, counters, status, st);
}

}  // namespace qr
