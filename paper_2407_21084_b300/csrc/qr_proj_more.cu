// qr_proj_more.cu -- projection tiles for the further index sets of the
// multi-instance engine (compiled apart to keep build times parallel).
#include "qr_ptree.cuh"

namespace qr {

#define QR_PROJ_MORE(X) \
    X(QR_G_L1, 3, 5)    \
    X(QR_G_L1, 5, 4)    \
    X(QR_G_L1, 6, 3)    \
    X(QR_G_L1, 6, 4)    \
    X(QR_G_L1, 7, 3)    \
    X(QR_G_L1, 8, 3)

int proj_tree_nodes_more(int kind, int d, int n)
{
#define QR_X(K, DD, NNN) \
    if (kind == K && d == DD && n == NNN) return FullTree<DD, NNN, K>::n;
    QR_PROJ_MORE(QR_X)
#undef QR_X
    return 0;
}

cudaError_t launch_project_tree_more(int prec, int kind, int n, const QrParams& P, const void* S, const int* perm,
                                     double2* partial, int i_lo, int i_hi, cudaStream_t st)
{
#define QR_X(K, DD, NNN)                                                                               \
    if (kind == K && P.d == DD && n == NNN)                                                            \
        return prec == QR_FP32 ? project_tree_t<float, DD, NNN, K>(P, S, perm, partial, i_lo, i_hi, st) \
                               : project_tree_t<double, DD, NNN, K>(P, S, perm, partial, i_lo, i_hi, st);
    QR_PROJ_MORE(QR_X)
#undef QR_X
    return cudaErrorInvalidValue;
}

}  // namespace qr
