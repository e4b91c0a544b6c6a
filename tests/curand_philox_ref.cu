// Reference outputs of cuRAND's Philox4_32_10 device generator, used only by
// tests/test_gpu_curand.py as an external known-answer source: for each row
// (seed, subsequence, offset) the first four words after curand_init, i.e.
// Philox4x32-10 at counter (offset/4, subsequence) and key seed.
#include <curand_kernel.h>

__global__ void k_curand_first4(const unsigned long long* __restrict__ rows, int n, uint4* __restrict__ out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    curandStatePhilox4_32_10_t st;
    curand_init(rows[3 * t], rows[3 * t + 1], rows[3 * t + 2], &st);
    out[t] = curand4(&st);
}

extern "C" int curand_first4(const unsigned long long* rows_host, int n, unsigned int* out_host)
{
    unsigned long long* d_rows = nullptr;
    uint4* d_out = nullptr;
    if (cudaMalloc(&d_rows, sizeof(unsigned long long) * 3 * n) != cudaSuccess) return 1;
    if (cudaMalloc(&d_out, sizeof(uint4) * n) != cudaSuccess) return 2;
    cudaMemcpy(d_rows, rows_host, sizeof(unsigned long long) * 3 * n, cudaMemcpyHostToDevice);
    k_curand_first4<<<(n + 127) / 128, 128>>>(d_rows, n, d_out);
    cudaError_t e = cudaMemcpy(out_host, d_out, sizeof(uint4) * n, cudaMemcpyDeviceToHost);
    cudaFree(d_rows);
    cudaFree(d_out);
    return e == cudaSuccess ? 0 : 3;
}
