// Measured throughput of the pipes the non-tensor parts of the hot path run
// on, for their roofline fractions: the 64-bit XOR + popcount that every
// sample-aware sweep test is made of (the mask test of Alg. 2 and of the pair
// sweep), plain 32-bit integer ALU work, and FP64 / FP32 fused multiply-add
// (the plain FP64 path and the FP32 CUDA-core path).  Each is a register-only
// loop kernel with eight independent chains per thread, launched over every
// SM and timed with CUDA events on the caller's stream (best of three after
// one warm-up launch).  Instrumentation, not part of the method: nothing here
// reads or changes a clock or any other device setting.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace nnqs {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

// XOR + 64-bit popcount per chain and step (the sweep's test); the
// accumulated counts are stored so that nothing is dead code
__global__ void __launch_bounds__(kPeakThreads) k_peak_popc(uint64_t seed, int iters, unsigned *__restrict__ sink) {
    const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    uint64_t x[kChains];
    unsigned acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        x[c] = (seed ^ (t * 0x9E3779B97F4A7C15ull)) + 0x632BE59BD9B4E019ull * (c + 1);
        acc[c] = 0;
    }
    uint64_t y = seed * 0xC2B2AE3D27D4EB4Full + t;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] += __popcll(x[c] ^ y);
        y = (y << 1) | (y >> 63);  // a new operand every step (one funnel shift per 8 tests)
    }
    unsigned s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    sink[t] = s;
}

// two 32-bit ALU operations per chain and step: a three-input logic op and
// an add
__global__ void __launch_bounds__(kPeakThreads) k_peak_int(uint32_t seed, int iters, unsigned *__restrict__ sink) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed ^ (t * 2654435761u) ^ (c * 40503u);
    const uint32_t k1 = seed | 1u, k2 = seed * 3u + 7u;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = ((a[c] ^ k1) & (a[c] | k2)) + a[(c + 1) % kChains];
    }
    unsigned s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s ^= a[c];
    sink[t] = s;
}

template <class T>
__global__ void __launch_bounds__(kPeakThreads) k_peak_fma(T seed, int iters, T *__restrict__ sink) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    T v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = seed + T(0.001) * T(t % 97) + T(c);
    const T m = T(0.999999), a = T(1e-7);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], m, a);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    sink[t] = s;
}

// best-of-three time of one kernel launch (ms), after a warm-up launch
template <class F>
nnqs_status time_best(cudaStream_t s, F launch, float *best_ms) {
    cudaEvent_t e0, e1;
    NNQS_CUDA_TRY(cudaEventCreate(&e0));
    NNQS_CUDA_TRY(cudaEventCreate(&e1));
    NNQS_TRY(launch());
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) {
        NNQS_CUDA_TRY(cudaEventRecord(e0, s));
        NNQS_TRY(launch());
        NNQS_CUDA_TRY(cudaEventRecord(e1, s));
        NNQS_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        NNQS_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *best_ms = best;
    return NNQS_OK;
}

}  // namespace
}  // namespace nnqs

using namespace nnqs;

extern "C" size_t nnqs_measure_peaks_sink_size(void) { return size_t(8 * num_sms()) * kPeakThreads * sizeof(double); }

extern "C" nnqs_status nnqs_measure_peaks(double out[4], void *sink, size_t sink_bytes, nnqs_stream stream) {
    if (!out || !sink) return set_error(NNQS_E_INVAL, "null argument");
    const int blocks = 8 * num_sms();  // 8 CTAs of 256 threads per SM
    const size_t threads = size_t(blocks) * kPeakThreads;
    if (sink_bytes < threads * sizeof(double))
        return set_error(NNQS_E_WORKSPACE, "peak kernels: sink needs " + std::to_string(threads * sizeof(double)) +
                                               " bytes");
    cudaStream_t s = (cudaStream_t)stream;
    float ms = 0.f;
    const int it_popc = 4096, it_int = 16384, it_d = 1024, it_f = 65536;
    unsigned *su = static_cast<unsigned *>(sink);
    NNQS_TRY(time_best(s, [&] { NNQS_LAUNCH("k_peak", s, k_peak_popc<<<blocks, kPeakThreads, 0, s>>>(0x1234567ull, it_popc, su)); return NNQS_OK; }, &ms));
    out[0] = double(threads) * it_popc * kChains / (ms * 1e-3);
    NNQS_TRY(time_best(s, [&] { NNQS_LAUNCH("k_peak", s, k_peak_int<<<blocks, kPeakThreads, 0, s>>>(0x9abcdefu, it_int, su)); return NNQS_OK; }, &ms));
    out[1] = 2.0 * double(threads) * it_int * kChains / (ms * 1e-3);
    double *sd = static_cast<double *>(sink);
    NNQS_TRY(time_best(s, [&] { NNQS_LAUNCH("k_peak", s, k_peak_fma<double><<<blocks, kPeakThreads, 0, s>>>(1.0, it_d, sd)); return NNQS_OK; }, &ms));
    out[2] = 2.0 * double(threads) * it_d * kChains / (ms * 1e-3);
    float *sf = static_cast<float *>(sink);
    NNQS_TRY(time_best(s, [&] { NNQS_LAUNCH("k_peak", s, k_peak_fma<float><<<blocks, kPeakThreads, 0, s>>>(1.0f, it_f, sf)); return NNQS_OK; }, &ms));
    out[3] = 2.0 * double(threads) * it_f * kChains / (ms * 1e-3);
    return NNQS_OK;
}
