// Measured integer-ALU rates of this device: the denominators of the tuple
// kernel's roofline (its work is 32-bit population counts and three-input
// logic operations on candidate masks). Not part of the paper's method.
//
// Each thread runs eight independent dependency chains so that the SM's
// issue slots, not instruction latency, bound the rate; the chains' results
// are stored so that the compiler keeps every operation.
#include "sbc_internal.cuh"

namespace sbc {
namespace {

constexpr int PK_THREADS = 256;
constexpr int PK_CHAINS = 8;

// Per chain and iteration: one POPC (plus the XOR and IADD that feed and
// consume it, on other pipes).
__global__ void __launch_bounds__(PK_THREADS) k_popc_rate(uint32_t seed, int iters, uint32_t *out) {
    uint32_t x[PK_CHAINS], acc[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; c++) {
        x[c] = seed * (threadIdx.x + 1) + 0x9E3779B9u * (c + 1) + blockIdx.x;
        acc[c] = 0;
    }
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int c = 0; c < PK_CHAINS; c++) {
            acc[c] += __popc(x[c] ^ (uint32_t)it);
            x[c] += acc[c];
        }
    }
    uint32_t s = 0;
#pragma unroll
    for (int c = 0; c < PK_CHAINS; c++) s ^= acc[c] + x[c];
    out[blockIdx.x * PK_THREADS + threadIdx.x] = s;
}

// Per chain and iteration: one three-input logic operation.
__global__ void __launch_bounds__(PK_THREADS) k_lop3_rate(uint32_t seed, int iters, uint32_t *out) {
    uint32_t x[PK_CHAINS];
    const uint32_t y = seed ^ threadIdx.x;
#pragma unroll
    for (int c = 0; c < PK_CHAINS; c++) x[c] = seed * (threadIdx.x + 1) + 0x85EBCA6Bu * (c + 1);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int c = 0; c < PK_CHAINS; c++) {
            uint32_t r;
            asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(r) : "r"(x[c]), "r"(y), "r"((uint32_t)it));
            x[c] = r;
        }
    }
    uint32_t s = 0;
#pragma unroll
    for (int c = 0; c < PK_CHAINS; c++) s ^= x[c];
    out[blockIdx.x * PK_THREADS + threadIdx.x] = s;
}

}  // namespace

void measure_alu_rates(double *popc_per_s, double *lop3_per_s, cudaStream_t s) {
    int dev = 0, sms = 0, per_sm = 0;
    SBC_CUDA(cudaGetDevice(&dev));
    SBC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SBC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_popc_rate, PK_THREADS, 0));
    const int grid = sms * (per_sm > 0 ? per_sm : 1);
    const int iters = 1 << 14;
    DevBuf<uint32_t> out((size_t)grid * PK_THREADS, s);
    cudaEvent_t e0, e1;
    SBC_CUDA(cudaEventCreate(&e0));
    SBC_CUDA(cudaEventCreate(&e1));
    auto timed = [&](bool popc) -> double {
        float best = 3.0e38f;
        for (int rep = 0; rep < 4; rep++) {  // first launch warms up
            SBC_CUDA(cudaEventRecord(e0, s));
            if (popc) k_popc_rate<<<grid, PK_THREADS, 0, s>>>(0x12345u + rep, iters, out.ptr);
            else k_lop3_rate<<<grid, PK_THREADS, 0, s>>>(0x12345u + rep, iters, out.ptr);
            SBC_LAUNCHED();
            g_launches++;
            SBC_CUDA(cudaEventRecord(e1, s));
            SBC_CUDA(cudaEventSynchronize(e1));
            float ms = 0;
            SBC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0) best = ms < best ? ms : best;
        }
        const double ops = (double)grid * PK_THREADS * iters * PK_CHAINS;
        return ops / (best / 1000.0);
    };
    try {
        *popc_per_s = timed(true);
        *lop3_per_s = timed(false);
    } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
}

}  // namespace sbc

extern "C" sbc_status sbc_measure_alu_rates(double *popc_per_s, double *lop3_per_s, void *stream) {
    try {
        if (!popc_per_s || !lop3_per_s) sbc::fail(SBC_E_INVAL, "output pointers must not be NULL");
        sbc::measure_alu_rates(popc_per_s, lop3_per_s, (cudaStream_t)stream);
    } catch (const sbc::SbcError &e) {
        sbc::set_last_error(e.what());
        return e.status;
    } catch (const std::exception &e) {
        sbc::set_last_error(e.what());
        return SBC_E_CUDA;
    }
    return SBC_OK;
}
