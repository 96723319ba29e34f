// peaks.cu -- measured roofs of this GPU for the roofline of the Dslash and the CG phase:
// FP32 and FP64 fused multiply-add throughput, read bandwidth from L2 and from HBM, the
// time of one back-to-back kernel launch, and one grid-wide barrier of the persistent CG
// kernel (the same barrier code).  Not part of the paper's method: the measured ceilings the
// kernels' timings are compared with.
#include <cstring>

#include "cg_phase.cuh"

namespace hisq {

// each thread: C independent FMA chains of n steps (2 flops per FMA)
template <class R, int C>
__global__ void __launch_bounds__(256) k_peak_fma(int n, R a, R b, R *out)
{
    R v[C];
#pragma unroll
    for (int c = 0; c < C; c++) v[c] = (R)(threadIdx.x + c);
    for (int i = 0; i < n; i++) {
#pragma unroll
        for (int c = 0; c < C; c++) v[c] = v[c] * a + b;
    }
    R s = 0;
#pragma unroll
    for (int c = 0; c < C; c++) s += v[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// coalesced 16-byte loads through L2 (L1 bypassed), eight in flight per thread
__global__ void __launch_bounds__(256) k_peak_read(const uint4 *a, size_t n, unsigned *out)
{
    const size_t nt = (size_t)gridDim.x * blockDim.x, t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    unsigned acc = 0;
    for (size_t base = 0; base < n; base += 8 * nt) {
        uint4 v[8];
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const size_t i = base + j * nt + t;
            v[j] = i < n ? __ldcg(a + i) : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int j = 0; j < 8; j++) acc ^= v[j].x ^ v[j].w;
    }
    out[t] = acc;
}

__global__ void k_peak_empty(unsigned *out)
{
    if (out && threadIdx.x == 0 && blockIdx.x == 0) out[0] = 0u;
}

__global__ void __launch_bounds__(512) k_peak_barrier(PhaseSlot *slots, int n, DevStatus *st)
{
    for (int i = 0; i < n; i++)
        if (!grid_barrier(slots, (unsigned)(i + 1), nullptr, st, 1000000000ull)) return;
}

}  // namespace hisq

using namespace hisq;

extern "C" int hisq_measure_peaks(int device, hisq_peaks *out)
{
    if (!out) return HISQ_EINVAL;
    std::memset(out, 0, sizeof(*out));
    if (cudaSetDevice(device) != cudaSuccess) return HISQ_ECUDA;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const size_t l2_bytes = 64ull << 20, hbm_bytes = 2048ull << 20;
    void *buf = nullptr, *res = nullptr, *slots = nullptr;
    DevStatus *st = nullptr;
    const int blocks = 8 * sms, threads = 256;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&buf, hbm_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&res, sizeof(double) * blocks * threads);
    if (e == cudaSuccess) e = cudaMalloc(&slots, sizeof(PhaseSlot) * kPhaseMaxBlocks);
    if (e == cudaSuccess) e = cudaMalloc(&st, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMemset(buf, 0, hbm_bytes);
    if (e == cudaSuccess) e = cudaMemset(st, 0, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    auto time_ms = [&](auto &&launch, int reps) -> double {
        launch();
        cudaEventRecord(e0);
        for (int r = 0; r < reps; r++) launch();
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms / reps;
    };
    if (e == cudaSuccess) {
        // long enough (tens of ms) for the clocks and pipes to settle
        const int n = 65536;
        double ms = time_ms([&] { k_peak_fma<float, 8><<<blocks, threads>>>(n, 0.999f, 0.5f, (float *)res); }, 5);
        out->fp32_tflops = 2.0 * 8 * n * (double)blocks * threads / (ms * 1e-3) / 1e12;
        const int nd = 2048;
        ms = time_ms([&] { k_peak_fma<double, 16><<<blocks, threads>>>(nd, 0.999, 0.5, (double *)res); }, 5);
        out->fp64_tflops = 2.0 * 16 * nd * (double)blocks * threads / (ms * 1e-3) / 1e12;
        const int rb = 4 * sms;
        ms = time_ms([&] { k_peak_read<<<rb, threads>>>((const uint4 *)buf, l2_bytes / 16, (unsigned *)res); }, 20);
        // the empty launch of the same shape is subtracted: a single pass over 64 MB is short
        const double empty = time_ms([&] { k_peak_read<<<rb, threads>>>((const uint4 *)buf, 0, (unsigned *)res); }, 20);
        out->l2_read_gbs = (double)l2_bytes / ((ms - empty) * 1e-3) / 1e9;
        ms = time_ms([&] { k_peak_read<<<rb, threads>>>((const uint4 *)buf, hbm_bytes / 16, (unsigned *)res); }, 10);
        out->hbm_read_gbs = (double)hbm_bytes / (ms * 1e-3) / 1e9;
        out->launch_us = 1e3 * time_ms([&] { k_peak_empty<<<rb, threads>>>(nullptr); }, 100);
        int coop = 0;
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device);
        if (coop && sms <= 512) {
            const int nb = 1000;
            cudaMemset(slots, 0, sizeof(PhaseSlot) * kPhaseMaxBlocks);
            PhaseSlot *sp = static_cast<PhaseSlot *>(slots);
            int nbar = nb;
            void *args[] = {&sp, &nbar, &st};
            cudaEventRecord(e0);
            e = cudaLaunchCooperativeKernel((void *)k_peak_barrier, dim3(sms), dim3(512), args, 0, 0);
            cudaEventRecord(e1);
            cudaEventSynchronize(e1);
            float bms = 0.f;
            cudaEventElapsedTime(&bms, e0, e1);
            out->grid_barrier_us = 1e3 * bms / nb;
        }
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        DevStatus h{};
        if (e == cudaSuccess) e = cudaMemcpy(&h, st, sizeof(h), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && h.error) out->grid_barrier_us = -1.0; // a wait ran out
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (buf) cudaFree(buf);
    if (res) cudaFree(res);
    if (slots) cudaFree(slots);
    if (st) cudaFree(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? HISQ_ENOMEM : HISQ_ECUDA;
    }
    return HISQ_OK;
}
