// qr_mlp.cu -- learned warm start: a small MLP mapping (PDE parameters, t_i)
// to the coefficient row alpha_i, trained and evaluated by the kernels of
// this file (tiled FP32 GEMM with fused bias/GELU epilogues, GELU backward,
// Adam). Not part of the paper: it replaces the y == 0 start of the Picard
// iteration by a prediction; the iteration itself is unchanged and corrects
// whatever error the prediction has.
//
// Layout: activations are row-major [batch x width]; a layer's weights W are
// row-major [n_in x n_out] (y = x W + b). All buffers are device memory owned
// by the qr_mlp object; inputs/targets are device pointers of the caller.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "qr_device.cuh"

struct qr_mlp {
    int n_layers = 0;             // weight layers
    std::vector<int> dims;        // n_layers + 1 sizes
    std::vector<size_t> w_off, b_off;
    size_t n_params = 0;
    float* d_params = nullptr;    // all W and b, flat
    float* d_grad = nullptr;
    float* d_m = nullptr;         // Adam moments
    float* d_v = nullptr;
    float* d_act = nullptr;       // pre-activations and activations of the last batch
    float* d_dact = nullptr;
    float* d_loss = nullptr;
    int cap_batch = 0;
    long long step = 0;
    cudaStream_t stream = nullptr;
    std::string err;
};

namespace {

constexpr int TM = 64, TN = 64, TK = 16;

// C[M x N] = op(A)[M x K] op(B)[K x N] (+ bias, + GELU), op = optional transpose.
// A is [M x K] row-major (lda) or, transposed, [K x M]; B likewise.
// epi: 0 = plain, 1 = +bias, 2 = +bias then GELU (pre-activation saved to Z).
__global__ void __launch_bounds__(256) k_gemm(const float* __restrict__ A, const float* __restrict__ B,
                                              float* __restrict__ C, int M, int N, int K, int lda, int ldb,
                                              int ldc, int ta, int tb, const float* __restrict__ bias, int epi,
                                              float* __restrict__ Z, float beta)
{
    __shared__ float As[TK][TM + 4];
    __shared__ float Bs[TK][TN + 4];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int row0 = blockIdx.y * TM, col0 = blockIdx.x * TN;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += TK) {
        for (int t = threadIdx.x; t < TM * TK; t += 256) {
            const int r = t / TK, kk = t % TK;
            const int gr = row0 + r, gk = k0 + kk;
            float v = 0.f;
            if (gr < M && gk < K) v = ta ? A[(size_t)gk * lda + gr] : A[(size_t)gr * lda + gk];
            As[kk][r] = v;
        }
        for (int t = threadIdx.x; t < TK * TN; t += 256) {
            const int kk = t / TN, c = t % TN;
            const int gk = k0 + kk, gc = col0 + c;
            float v = 0.f;
            if (gk < K && gc < N) v = tb ? B[(size_t)gc * ldb + gk] : B[(size_t)gk * ldb + gc];
            Bs[kk][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = As[kk][ty * 4 + q];
                b[q] = Bs[kk][tx * 4 + q];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int r = row0 + ty * 4 + p;
        if (r >= M) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c = col0 + tx * 4 + q;
            if (c >= N) continue;
            float v = acc[p][q];
            if (epi >= 1) v += bias[c];
            if (epi == 2) {
                Z[(size_t)r * ldc + c] = v;
                v = 0.5f * v * (1.0f + erff(v * 0.70710678118654752f));
            }
            float* out = C + (size_t)r * ldc + c;
            *out = beta != 0.f ? beta * *out + v : v;
        }
    }
}

// dZ = dH * gelu'(Z)
__global__ void k_gelu_back(const float* __restrict__ Z, float* __restrict__ dH, long long n)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float z = Z[t];
    const float cdf = 0.5f * (1.0f + erff(z * 0.70710678118654752f));
    const float pdf = 0.39894228040143268f * expf(-0.5f * z * z);
    dH[t] *= cdf + z * pdf;
}

// column sums of dY [M x N] -> db (bias gradient), fixed order
__global__ void k_colsum(const float* __restrict__ dY, int M, int N, float* __restrict__ db)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    float s = 0.f;
    for (int r = 0; r < M; ++r) s += dY[(size_t)r * N + c];
    db[c] = s;
}

// dY = (Y - T) * 2/(B*n_out); per-block partial squared error into loss[blockIdx.x]
__global__ void k_mse_grad(const float* __restrict__ Y, const float* __restrict__ T, float* __restrict__ dY,
                           long long n, float scale, float* __restrict__ loss_part)
{
    __shared__ float red[256];
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float e = 0.f;
    if (t < n) {
        const float r = Y[t] - T[t];
        dY[t] = 2.0f * scale * r;
        e = r * r;
    }
    red[threadIdx.x] = e;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_part[blockIdx.x] = red[0];
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float gt = g[t];
    const float mt = b1 * m[t] + (1.f - b1) * gt;
    const float vt = b2 * v[t] + (1.f - b2) * gt * gt;
    m[t] = mt;
    v[t] = vt;
    p[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
}

// deterministic initialisation: uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) from Philox
__global__ void k_init(float* __restrict__ w, long long n, float scale, uint32_t key0, uint32_t key1, uint32_t tagc)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const uint4 c = qr::philox4x32_10(make_uint4((uint32_t)t, (uint32_t)(t >> 32), tagc, 0x4d4c5000u),
                                      make_uint2(key0, key1));
    w[t] = scale * (2.0f * ((float)(c.x >> 8) * 0x1p-24f) - 1.0f);
}

cudaError_t gemm(const float* A, const float* B, float* C, int M, int N, int K, int lda, int ldb, int ldc, int ta,
                 int tb, const float* bias, int epi, float* Z, float beta, cudaStream_t st)
{
    dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM);
    k_gemm<<<grid, 256, 0, st>>>(A, B, C, M, N, K, lda, ldb, ldc, ta, tb, bias, epi, Z, beta);
    return cudaGetLastError();
}

qr_status mfail(qr_mlp* m, qr_status s, const std::string& msg)
{
    if (m) m->err = msg;
    return s;
}

// activation buffers: for layer l (0..L-1): Z_l (pre-activation, hidden layers)
// and H_{l+1} (output of layer l); H_0 = the input (caller memory).
struct ActView {
    float* Z[16];
    float* H[17];
};

ActView act_view(qr_mlp* m, const float* X, int B)
{
    ActView v{};
    v.H[0] = const_cast<float*>(X);
    float* p = m->d_act;
    for (int l = 0; l < m->n_layers; ++l) {
        v.Z[l] = p;
        p += (size_t)B * m->dims[l + 1];
        v.H[l + 1] = p;
        p += (size_t)B * m->dims[l + 1];
    }
    return v;
}

qr_status forward(qr_mlp* m, const float* X, int B, float* Y_out)
{
    ActView v = act_view(m, X, B);
    for (int l = 0; l < m->n_layers; ++l) {
        const int ni = m->dims[l], no = m->dims[l + 1];
        const bool last = l + 1 == m->n_layers;
        float* out = last && Y_out ? Y_out : v.H[l + 1];
        cudaError_t e = gemm(v.H[l], m->d_params + m->w_off[l], out, B, no, ni, ni, no, no, 0, 0,
                             m->d_params + m->b_off[l], last ? 1 : 2, v.Z[l], 0.f, m->stream);
        if (e != cudaSuccess) return mfail(m, QR_ECUDA, cudaGetErrorString(e));
        if (last && Y_out && out != v.H[l + 1])
            cudaMemcpyAsync(v.H[l + 1], out, sizeof(float) * (size_t)B * no, cudaMemcpyDeviceToDevice, m->stream);
    }
    return QR_OK;
}

// gradients of the mean squared error into d_grad; loss (host) optional
qr_status backward(qr_mlp* m, const float* X, const float* T, int B, float* loss_out)
{
    ActView v = act_view(m, X, B);
    const int L = m->n_layers;
    const int nout = m->dims[L];
    const long long n = (long long)B * nout;
    const int nb = (int)((n + 255) / 256);
    float* dY = m->d_dact;  // [B x max_width] scratch, two halves
    const size_t half = (size_t)m->cap_batch * (size_t)*std::max_element(m->dims.begin(), m->dims.end());
    float* dA = dY;
    float* dB_ = dY + half;
    k_mse_grad<<<nb, 256, 0, m->stream>>>(v.H[L], T, dA, n, 1.0f / (float)n, m->d_loss);
    for (int l = L - 1; l >= 0; --l) {
        const int ni = m->dims[l], no = m->dims[l + 1];
        // dW_l = H_l^T dZ_l ; db_l = colsum(dZ_l)
        cudaError_t e = gemm(v.H[l], dA, m->d_grad + m->w_off[l], ni, no, B, ni, no, no, 1, 0, nullptr, 0, nullptr,
                             0.f, m->stream);
        if (e != cudaSuccess) return mfail(m, QR_ECUDA, cudaGetErrorString(e));
        k_colsum<<<(no + 255) / 256, 256, 0, m->stream>>>(dA, B, no, m->d_grad + m->b_off[l]);
        if (l > 0) {
            // dH_l = dZ_l W_l^T, then through GELU of layer l-1
            e = gemm(dA, m->d_params + m->w_off[l], dB_, B, ni, no, no, no, ni, 0, 1, nullptr, 0, nullptr, 0.f,
                     m->stream);
            if (e != cudaSuccess) return mfail(m, QR_ECUDA, cudaGetErrorString(e));
            const long long nh = (long long)B * ni;
            k_gelu_back<<<(unsigned)((nh + 255) / 256), 256, 0, m->stream>>>(v.Z[l - 1], dB_, nh);
            std::swap(dA, dB_);
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return mfail(m, QR_ECUDA, cudaGetErrorString(e));
    if (loss_out) {
        std::vector<float> parts(nb);
        cudaMemcpyAsync(parts.data(), m->d_loss, sizeof(float) * nb, cudaMemcpyDeviceToHost, m->stream);
        if (cudaStreamSynchronize(m->stream) != cudaSuccess) return mfail(m, QR_ECUDA, "sync");
        double s = 0;
        for (float p : parts) s += p;
        *loss_out = (float)(s / (double)n);
    }
    return QR_OK;
}

}  // namespace

extern "C" {

qr_status qr_mlp_create(qr_mlp** out, int n_in, int width, int depth, int n_out, int max_batch,
                        unsigned long long seed, void* stream)
{
    if (!out) return QR_EINVAL;
    *out = nullptr;
    if (n_in < 1 || width < 1 || depth < 1 || depth > 14 || n_out < 1 || max_batch < 1) return QR_EINVAL;
    qr_mlp* m = new (std::nothrow) qr_mlp();
    if (!m) return QR_ENOMEM;
    m->stream = static_cast<cudaStream_t>(stream);
    m->dims.push_back(n_in);
    for (int h = 0; h < depth; ++h) m->dims.push_back(width);
    m->dims.push_back(n_out);
    m->n_layers = depth + 1;
    for (int l = 0; l < m->n_layers; ++l) {
        m->w_off.push_back(m->n_params);
        m->n_params += (size_t)m->dims[l] * m->dims[l + 1];
        m->b_off.push_back(m->n_params);
        m->n_params += (size_t)m->dims[l + 1];
    }
    m->cap_batch = max_batch;
    size_t act = 0;
    for (int l = 0; l < m->n_layers; ++l) act += 2 * (size_t)max_batch * m->dims[l + 1];
    const size_t wmax = (size_t)*std::max_element(m->dims.begin(), m->dims.end());
    bool ok = cudaMalloc(&m->d_params, 4 * m->n_params) == cudaSuccess &&
              cudaMalloc(&m->d_grad, 4 * m->n_params) == cudaSuccess &&
              cudaMalloc(&m->d_m, 4 * m->n_params) == cudaSuccess &&
              cudaMalloc(&m->d_v, 4 * m->n_params) == cudaSuccess && cudaMalloc(&m->d_act, 4 * act) == cudaSuccess &&
              cudaMalloc(&m->d_dact, 4 * 2 * (size_t)max_batch * wmax) == cudaSuccess &&
              cudaMalloc(&m->d_loss, 4 * (((size_t)max_batch * n_out + 255) / 256 + 1)) == cudaSuccess;
    if (!ok) {
        *out = m;
        m->err = "device allocation failed";
        return QR_ENOMEM;
    }
    cudaMemsetAsync(m->d_m, 0, 4 * m->n_params, m->stream);
    cudaMemsetAsync(m->d_v, 0, 4 * m->n_params, m->stream);
    for (int l = 0; l < m->n_layers; ++l) {
        const long long nw = (long long)m->dims[l] * m->dims[l + 1];
        const float sc = 1.0f / std::sqrt((float)m->dims[l]);
        k_init<<<(unsigned)((nw + 255) / 256), 256, 0, m->stream>>>(m->d_params + m->w_off[l], nw, sc,
                                                                     (uint32_t)seed, (uint32_t)(seed >> 32),
                                                                     (uint32_t)l);
        cudaMemsetAsync(m->d_params + m->b_off[l], 0, 4 * (size_t)m->dims[l + 1], m->stream);
    }
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) {
        *out = m;
        m->err = "initialisation failed";
        return QR_ECUDA;
    }
    *out = m;
    return QR_OK;
}

long long qr_mlp_num_params(const qr_mlp* m) { return m ? (long long)m->n_params : -1; }

qr_status qr_mlp_get_params(const qr_mlp* m, float* out)
{
    if (!m || !out) return QR_EINVAL;
    // ordered after the work queued on the network's stream
    if (cudaMemcpyAsync(out, m->d_params, 4 * m->n_params, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess)
        return QR_ECUDA;
    return QR_OK;
}

qr_status qr_mlp_set_params(qr_mlp* m, const float* in)
{
    if (!m || !in) return QR_EINVAL;
    if (cudaMemcpyAsync(m->d_params, in, 4 * m->n_params, cudaMemcpyHostToDevice, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess)
        return QR_ECUDA;
    return QR_OK;
}

qr_status qr_mlp_forward(qr_mlp* m, const float* X, int B, float* Y)
{
    if (!m || !X || !Y || B < 1 || B > m->cap_batch) return mfail(m, QR_EINVAL, "qr_mlp_forward: bad arguments");
    qr_status s = forward(m, X, B, Y);
    if (s != QR_OK) return s;
    return cudaStreamSynchronize(m->stream) == cudaSuccess ? QR_OK : mfail(m, QR_ECUDA, "sync");
}

qr_status qr_mlp_gradients(qr_mlp* m, const float* X, const float* T, int B, float* grad_out, float* loss_out)
{
    if (!m || !X || !T || B < 1 || B > m->cap_batch) return mfail(m, QR_EINVAL, "qr_mlp_gradients: bad arguments");
    qr_status s = forward(m, X, B, nullptr);
    if (s == QR_OK) s = backward(m, X, T, B, loss_out);
    if (s != QR_OK) return s;
    if (grad_out && (cudaMemcpyAsync(grad_out, m->d_grad, 4 * m->n_params, cudaMemcpyDeviceToHost, m->stream) !=
                         cudaSuccess ||
                     cudaStreamSynchronize(m->stream) != cudaSuccess))
        return mfail(m, QR_ECUDA, "copy gradients");
    return QR_OK;
}

qr_status qr_mlp_train_step(qr_mlp* m, const float* X, const float* T, int B, float lr, float* loss_out)
{
    if (!m || !X || !T || B < 1 || B > m->cap_batch || !(lr > 0.f))
        return mfail(m, QR_EINVAL, "qr_mlp_train_step: bad arguments");
    qr_status s = forward(m, X, B, nullptr);
    if (s == QR_OK) s = backward(m, X, T, B, loss_out);
    if (s != QR_OK) return s;
    m->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
    const long long n = (long long)m->n_params;
    k_adam<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(m->d_params, m->d_grad, m->d_m, m->d_v, n, lr, b1, b2,
                                                                1e-8f, c1, c2);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? QR_OK : mfail(m, QR_ECUDA, cudaGetErrorString(e));
}

const char* qr_mlp_last_error(const qr_mlp* m) { return m ? m->err.c_str() : "no network"; }

void qr_mlp_destroy(qr_mlp* m)
{
    if (!m) return;
    float* ptrs[] = {m->d_params, m->d_grad, m->d_m, m->d_v, m->d_act, m->d_dact, m->d_loss};
    for (float* p : ptrs)
        if (p) cudaFree(p);
    delete m;
}

}  // extern "C"
