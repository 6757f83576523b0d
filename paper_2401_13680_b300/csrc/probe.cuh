// Measured arithmetic rates of the device, for the roofline of an ALU-bound
// kernel (no counterpart in the paper): fused multiply-adds in FP32 and in
// FP64, eight independent dependency chains per thread, enough warps to fill
// every scheduler.
#pragma once

namespace pastila {

constexpr int PROBE_CHAINS = 8;

template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(T* __restrict__ out, int iters, T seed) {
    T a[PROBE_CHAINS];
#pragma unroll
    for (int j = 0; j < PROBE_CHAINS; ++j) a[j] = seed + (T)(threadIdx.x & 31) * (T)1e-3 + (T)j;
    const T b = (T)0.9999999, c = (T)1e-7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int j = 0; j < PROBE_CHAINS; ++j) a[j] = fma(a[j], b, c);
        }
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < PROBE_CHAINS; ++j) s += a[j];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace pastila
