// qr_static.cu -- projection of given responses with no device allocation.
//
// qr_project_static runs the same projection kernel as qr_picard_step on
// responses the caller supplies, but keeps the per-CTA FP64 partial sums in
// a fixed array compiled into the library instead of memory the context
// allocates, so that a caller who cannot allocate device memory at the time
// of the call can still run it.
#include <cstdio>
#include <mutex>

#include "qr_fast.h"
#include "qr_internal.h"

namespace {

constexpr size_t kPartialSlots = size_t(1) << 20;  // double2 slots: 16 MiB
constexpr int kMaxDevices = 64;

// Scratch for the per-CTA partial sums, one copy per GPU that loads the
// library, held until the process exits. Host code must not pass the symbol
// itself to a kernel: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) double2 g_partials[kPartialSlots];

std::mutex g_mu;
double2* g_addr[kMaxDevices] = {};

// device address of g_partials on device `dev` (the context's device),
// looked up once per device with that device current; the caller's current
// device is restored afterwards
cudaError_t scratch_address(int dev, double2** out)
{
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        int cur = 0;
        cudaError_t e = cudaGetDevice(&cur);
        if (e != cudaSuccess) return e;
        if (cur != dev && (e = cudaSetDevice(dev)) != cudaSuccess) return e;
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_partials);
        if (cur != dev) {
            const cudaError_t e2 = cudaSetDevice(cur);
            if (e == cudaSuccess) e = e2;
        }
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<double2*>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

__global__ void k_reduce_rows(const double2* __restrict__ partial, int n_chunks, int nGp, long long M, int nG,
                              int zero_idx, int rows, double2* __restrict__ out)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)rows * nGp) return;
    const int r = (int)(idx / nGp), e = (int)(idx % nGp);
    const double2* p = partial + (size_t)r * n_chunks * nGp + e;
    double sx = 0.0, sy = 0.0;
    for (int c = 0; c < n_chunks; ++c) {
        const double2 v = p[(size_t)c * nGp];
        sx += v.x;
        sy += v.y;
    }
    sx /= (double)M;
    sy /= (double)M;
    if (e == 0) sy = 0.0;
    double2* row = out + (size_t)r * nG;
    row[zero_idx + e] = make_double2(sx, sy);
    if (e > 0) row[zero_idx - e] = make_double2(sx, -sy);
}

}  // namespace

extern "C" qr_status qr_project_static(qr_ctx* ctx, const void* S, int i_lo, int i_hi, double* alpha_out)
{
    qr::CtxView v{};
    if (!qr::ctx_view(ctx, &v)) return QR_EINVAL;
    if (!S || !alpha_out || i_lo < 0 || i_hi > v.N || i_hi <= i_lo) {
        qr::ctx_set_error(ctx, "qr_project_static: bad arguments");
        return QR_EINVAL;
    }
    const qr::QrParams& P = *v.P;
    if (v.sharded) {
        qr::ctx_set_error(ctx, "qr_project_static: not for a sharded context");
        return QR_EINVAL;
    }
    if (P.half_angle) {
        qr::ctx_set_error(ctx, "qr_project_static: the cosine basis is not supported");
        return QR_ENOTIMPL;
    }
    const size_t need = (size_t)(i_hi - i_lo) * (size_t)P.n_chunks * (size_t)P.nGp;
    if (need > kPartialSlots) {
        char msg[200];
        std::snprintf(msg, sizeof msg,
                      "qr_project_static: %zu partial sums needed, the fixed scratch holds %zu "
                      "(rows x chunks x |Gamma_+|); project fewer rows per call",
                      need, kPartialSlots);
        qr::ctx_set_error(ctx, msg);
        return QR_EINVAL;
    }
    // the context's device is current for the call (its stream and buffers
    // live there); the caller's current device is restored on return
    int cur = 0;
    cudaError_t e = cudaGetDevice(&cur);
    if (e == cudaSuccess && cur != v.device) e = cudaSetDevice(v.device);
    if (e != cudaSuccess) {
        qr::ctx_set_error(ctx, cudaGetErrorString(e));
        return QR_ECUDA;
    }
    struct Restore {
        int dev;
        bool on;
        ~Restore()
        {
            if (on) (void)cudaSetDevice(dev);
        }
    } restore{cur, cur != v.device};
    double2* scratch = nullptr;
    e = scratch_address(v.device, &scratch);
    // the same projection kernel qr_picard_step runs for this context: the
    // compiled tiled projection when one covers the index set, else the
    // table-driven one; both write every partial slot of the rows they cover
    if (e == cudaSuccess)
        e = v.proj_nodes ? qr::launch_project_tree(v.prec, v.gkind, v.gn, P, S, v.perm, scratch, i_lo, i_hi, v.stream)
                         : qr::launch_project(v.prec, P, v.tab, v.first, S, scratch, i_lo, i_hi, v.stream);
    if (e == cudaSuccess) {
        const long long total = (long long)(i_hi - i_lo) * P.nGp;
        k_reduce_rows<<<(unsigned)((total + 255) / 256), 256, 0, v.stream>>>(
            scratch, P.n_chunks, P.nGp, P.M, v.nG, v.zero_idx, i_hi - i_lo,
            reinterpret_cast<double2*>(alpha_out));
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        qr::ctx_set_error(ctx, cudaGetErrorString(e));
        return QR_ECUDA;
    }
    return QR_OK;
}
