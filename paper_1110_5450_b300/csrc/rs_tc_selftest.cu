// rs_tc_selftest.cu -- a one-CTA tcgen05 GEMM on host-given matrices, used to
// check the tensor-core building blocks (shared-memory layouts, descriptors,
// tensor-memory accumulators) against a CPU product.  Every wait is bounded
// and the tensor memory is freed on every path.
#include <cstring>
#include <string>

#include "rs_internal.h"
#include "rs_tc.cuh"

namespace rs {
namespace {

constexpr int kTcThreads = 128;
constexpr size_t kRegion = 96 * 1024; // room for A and for B (generous: a wrong stride stays inside)

__device__ __forceinline__ uint64_t now_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void __launch_bounds__(kTcThreads) tc_gemm_test_kernel(const uint16_t *A, const uint16_t *B, float *D,
                                                                   int m, int n, int k, int a_mn, int b_mn,
                                                                   int variant, int bf16, int *err)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *sa = sm;
    unsigned char *sb = sm + kRegion;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + 2 * kRegion);
    uint32_t *slot = reinterpret_cast<uint32_t *>(sm + 2 * kRegion + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // operand strides of the canonical layout
    const uint32_t a_sk = a_mn ? uint32_t(m / 8) * 128u : 128u, a_sr = a_mn ? 128u : uint32_t(k / 8) * 128u;
    const uint32_t b_sk = b_mn ? uint32_t(n / 8) * 128u : 128u, b_sr = b_mn ? 128u : uint32_t(k / 8) * 128u;
    for (int e = tid; e < m * k; e += kTcThreads) {
        const int r = e / k, kk = e - r * k;
        *reinterpret_cast<uint16_t *>(sa + tc::canon_offset(a_mn, r, kk, a_sr, a_sk)) = A[e];
    }
    for (int e = tid; e < n * k; e += kTcThreads) {
        const int r = e / k, kk = e - r * k;
        *reinterpret_cast<uint16_t *>(sb + tc::canon_offset(b_mn, r, kk, b_sr, b_sk)) = B[e];
    }
    tc::fence_proxy_async();
    uint32_t ncols = 32;
    while (ncols < uint32_t(n)) ncols <<= 1;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::saddr(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tc::tmem_alloc(slot, ncols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *slot;

    if (tid == 0) {
        const uint32_t idesc = tc::idesc_f16(bf16 != 0, a_mn != 0, b_mn != 0, m, n);
        // leading / stride byte offsets: variant 0 encodes the K-direction
        // core-matrix stride as the leading offset and the row-direction (M or N)
        // stride as the stride offset; variant 1 swaps them
        const uint32_t a_lbo = variant ? a_sr : a_sk, a_sbo = variant ? a_sk : a_sr;
        const uint32_t b_lbo = variant ? b_sr : b_sk, b_sbo = variant ? b_sk : b_sr;
        for (int kb = 0; kb < k / 16; ++kb) {
            const uint64_t ad = tc::smem_desc(tc::saddr(sa) + uint32_t(kb) * 2u * a_sk, a_lbo, a_sbo);
            const uint64_t bd = tc::smem_desc(tc::saddr(sb) + uint32_t(kb) * 2u * b_sk, b_lbo, b_sbo);
            tc::mma_f16(taddr, ad, bd, idesc, kb > 0 ? 1u : 0u);
        }
        tc::mma_commit(bar);
    }
    // bounded wait for the MMAs (a correct run takes microseconds)
    bool ok = false;
    const uint64_t t0 = now_ns();
    for (uint32_t it = 0; it < (1u << 24); ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0, 20000;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(tc::saddr(bar))
            : "memory");
        if (done) {
            ok = true;
            break;
        }
        if (now_ns() - t0 > 2000000000ull) break;
    }
    tc::fence_after_sync();
    if (!ok) {
        if (tid == 0) atomicCAS(err, 0, 301);
    } else {
        for (int c0 = 0; c0 < n; c0 += 16) {
            uint32_t r[16];
            tc::tmem_ld16(taddr + (uint32_t(warp * 32) << 16) + uint32_t(c0), r);
            tc::tmem_ld_wait();
            const int row = warp * 32 + lane;
            for (int j = 0; j < 16 && c0 + j < n; ++j) D[size_t(row) * n + c0 + j] = __uint_as_float(r[j]);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, ncols);
}

} // namespace
} // namespace rs

using namespace rs;

extern "C" rs_status rs_tc_selftest(int32_t m, int32_t n, int32_t k, int32_t a_mn, int32_t b_mn, int32_t variant,
                                    int32_t bf16, const uint16_t *h_a, const uint16_t *h_b, float *h_d)
{
    // each operand's canonical layout (rows * k * 2 bytes) must fit its region
    if (m != 128 || n < 16 || n > 256 || n % 16 || k < 16 || k > 256 || k % 16 || !h_a || !h_b || !h_d ||
        size_t(m) * k * 2 > kRegion || size_t(n) * k * 2 > kRegion) {
        set_error("rs_tc_selftest: m = 128, n and k multiples of 16 up to 256, rows * k * 2 <= 96 KiB");
        return RS_ERR_INVALID_ARG;
    }
    uint16_t *da = nullptr, *db = nullptr;
    float *dd = nullptr;
    int *derr = nullptr;
    cudaError_t e = cudaMalloc(&da, size_t(m) * k * 2);
    if (e == cudaSuccess) e = cudaMalloc(&db, size_t(n) * k * 2);
    if (e == cudaSuccess) e = cudaMalloc(&dd, size_t(m) * n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&derr, 4);
    if (e == cudaSuccess) e = cudaMemset(derr, 0, 4);
    if (e == cudaSuccess) e = cudaMemset(dd, 0, size_t(m) * n * 4);
    if (e == cudaSuccess) e = cudaMemcpy(da, h_a, size_t(m) * k * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(db, h_b, size_t(n) * k * 2, cudaMemcpyHostToDevice);
    const size_t smem = 2 * kRegion + 64;
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_gemm_test_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e == cudaSuccess) {
        tc_gemm_test_kernel<<<1, kTcThreads, smem>>>(da, db, dd, m, n, k, a_mn, b_mn, variant, bf16, derr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&herr, derr, 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(h_d, dd, size_t(m) * n * 4, cudaMemcpyDeviceToHost);
    cudaFree(da);
    cudaFree(db);
    cudaFree(dd);
    cudaFree(derr);
    if (e != cudaSuccess) {
        set_error(std::string("rs_tc_selftest: ") + cudaGetErrorString(e));
        cudaGetLastError();
        return RS_ERR_CUDA;
    }
    if (herr) {
        set_error("rs_tc_selftest: the MMA completion wait ran out");
        return RS_ERR_TIMEOUT;
    }
    return RS_OK;
}
