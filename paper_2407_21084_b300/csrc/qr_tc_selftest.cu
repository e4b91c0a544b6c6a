// qr_tc_selftest.cu -- test hook for the tensor-core primitives of qr_tc.cuh:
// one 128 x 32 x 64 BF16 product through tcgen05.mma (operands staged in the
// 128-byte swizzled shared-memory layout, FP32 accumulator in tensor memory),
// read back with tcgen05.ld. It checks the descriptor encodings and the
// layouts the shared-point group kernel relies on against a product the
// caller computes on the host.
#include <cuda_runtime.h>

#include "qr_internal.h"
#include "qr_tc.cuh"

namespace qr {
namespace {

constexpr int kTM = 128, kTN = 32, kTK = 64;

__global__ void __launch_bounds__(kTM) k_tc_selftest(const uint16_t* __restrict__ A, const uint16_t* __restrict__ B,
                                                     float* __restrict__ D, unsigned* __restrict__ status)
{
    __shared__ __align__(1024) uint8_t sa[kTM * 128];
    __shared__ __align__(1024) uint8_t sb[kTN * 128];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5;
    // row tid of A (and of B for the first 32 threads), 8 BF16 per 16-byte chunk
#pragma unroll
    for (int k = 0; k < kTK; k += 8) {
        *reinterpret_cast<uint4*>(sa + sw128_offset(tid, k)) = *reinterpret_cast<const uint4*>(A + tid * kTK + k);
        if (tid < kTN)
            *reinterpret_cast<uint4*>(sb + sw128_offset(tid, k)) = *reinterpret_cast<const uint4*>(B + tid * kTK + k);
    }
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    // the swizzled tiles must start on 1024-byte shared addresses (checked,
    // not assumed: a misplaced tile would only give wrong products)
    const bool aligned = ((smem_u32(sa) | smem_u32(sb)) & 1023u) == 0;
    if (warp == 0) {
        tmem_alloc(&tslot, 32);
        tmem_relinquish();
    }
    fence_proxy_async_smem();  // the stores above, visible to the tensor core
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tslot;
    if (tid == 0 && aligned) {
        const uint32_t idesc = idesc_bf16_f32(kTM, kTN);
#pragma unroll
        for (int kk = 0; kk < kTK / 16; ++kk)
            tc_mma_bf16(tbase, sw128_desc(smem_u32(sa) + 32u * kk), sw128_desc(smem_u32(sb) + 32u * kk), idesc,
                        kk > 0);
        tc_commit(&bar);
    }
    const bool ok = __syncthreads_and(aligned && mbar_wait(&bar, 0));
    tc_fence_after();
    if (ok) {
        float v[32];
        tmem_ld_32x32(tbase + ((uint32_t)(warp * 32) << 16), v);
#pragma unroll
        for (int j = 0; j < kTN; ++j) D[tid * kTN + j] = v[j];
    } else if (tid == 0) {
        atomicOr(status, aligned ? ST_TIMEOUT : 2u);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tbase, 32);
}

}  // namespace
}  // namespace qr

extern "C" qr_status qr_tc_selftest(const uint16_t* A, const uint16_t* B, float* D)
{
    if (!A || !B || !D) return QR_EINVAL;
    uint16_t *dA = nullptr, *dB = nullptr;
    float* dD = nullptr;
    unsigned* dst = nullptr;
    qr_status s = QR_OK;
    do {
        if (cudaMalloc(&dA, sizeof(uint16_t) * qr::kTM * qr::kTK) != cudaSuccess ||
            cudaMalloc(&dB, sizeof(uint16_t) * qr::kTN * qr::kTK) != cudaSuccess ||
            cudaMalloc(&dD, sizeof(float) * qr::kTM * qr::kTN) != cudaSuccess ||
            cudaMalloc(&dst, sizeof(unsigned)) != cudaSuccess) {
            s = QR_ENOMEM;
            break;
        }
        if (cudaMemcpy(dA, A, sizeof(uint16_t) * qr::kTM * qr::kTK, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(dB, B, sizeof(uint16_t) * qr::kTN * qr::kTK, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemset(dst, 0, sizeof(unsigned)) != cudaSuccess || cudaMemset(dD, 0, sizeof(float) * qr::kTM * qr::kTN) != cudaSuccess) {
            s = QR_ECUDA;
            break;
        }
        qr::k_tc_selftest<<<1, qr::kTM>>>(dA, dB, dD, dst);
        unsigned st = 0;
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(&st, dst, sizeof st, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(D, dD, sizeof(float) * qr::kTM * qr::kTN, cudaMemcpyDeviceToHost) != cudaSuccess) {
            s = QR_ECUDA;
            break;
        }
        if (st & qr::ST_TIMEOUT) s = QR_ETIMEOUT;
        else if (st) s = QR_ECUDA;  // tiles not on 1024-byte shared addresses
    } while (false);
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dD);
    cudaFree(dst);
    return s;
}
