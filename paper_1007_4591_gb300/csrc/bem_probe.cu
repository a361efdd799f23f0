// FP32 throughput of the device the library runs on, for the near-field
// kernel's roofline: independent chains of packed FP32 fused multiply-adds
// (f32x2, the form the near-field kernel uses) on every SM, timed with CUDA
// events.  The derived peak (SMs x 128 lanes x 2 flop x clock) is the
// reference; this measures what the FMA pipe delivers.
#include "bem_internal.cuh"

namespace bem {

constexpr int PROBE_ITERS = 2048;
constexpr int PROBE_CHAINS = 4;

__global__ void k_ffma2_probe(float *out, float a, float b) {
    float2 x[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = make_float2((float)threadIdx.x + k, (float)threadIdx.x - k);
    const float2 A = make_float2(a, a), B = make_float2(b, b);
    for (int i = 0; i < PROBE_ITERS; ++i) {
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = __ffma2_rn(x[k], A, B);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += x[k].x + x[k].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

}  // namespace bem

using namespace bem;

extern "C" int bem_fp32_peak(double *tflops) {
    if (!tflops) {
        set_last_error("bem_fp32_peak: NULL");
        return BEM_EINVAL;
    }
    try {
        int dev = 0, nsm = 0;
        BEM_CUDA(cudaGetDevice(&dev));
        BEM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        const int threads = 256, blocks = nsm * 8;
        DArray<float> out;
        out.alloc((size_t)threads * blocks);
        cudaEvent_t a = nullptr, b = nullptr;
        BEM_CUDA(cudaEventCreate(&a));
        BEM_CUDA(cudaEventCreate(&b));
        double best = 0.0;
        for (int rep = 0; rep < 3; ++rep) {  // the first run warms the clocks up
            BEM_CUDA(cudaEventRecord(a, 0));
            k_ffma2_probe<<<blocks, threads>>>(out.p, 0.999f, 0.001f);
            BEM_CHECK_LAUNCH();
            BEM_CUDA(cudaEventRecord(b, 0));
            BEM_CUDA(cudaEventSynchronize(b));
            float ms = 0.f;
            BEM_CUDA(cudaEventElapsedTime(&ms, a, b));
            const double flop = 2.0 * 2.0 * PROBE_CHAINS * PROBE_ITERS * (double)threads * blocks;
            if (ms > 0.f) best = std::max(best, flop / (ms * 1e-3) / 1e12);
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        *tflops = best;
        return BEM_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.code;
    }
}
