// Order-preserving integer keys of floating-point values: a < b  <=>  key(a) < key(b)
// (for non-NaN values; -0 sorts just below +0).  Selections run on keys so that a
// bisection midpoint is an integer and every comparison is an integer compare.
#pragma once
#include <cstdint>

namespace pastila {

template <typename real> struct KeyOf;

template <> struct KeyOf<float> {
    typedef uint32_t type;
    static constexpr uint32_t TOP = 0x80000000u;
    __host__ __device__ static inline uint32_t enc(float f) {
#ifdef __CUDA_ARCH__
        uint32_t u = __float_as_uint(f);
#else
        uint32_t u;
        __builtin_memcpy(&u, &f, 4);
#endif
        return (u & TOP) ? ~u : (u | TOP);
    }
    __host__ __device__ static inline float dec(uint32_t k) {
        uint32_t u = (k & TOP) ? (k & ~TOP) : ~k;
#ifdef __CUDA_ARCH__
        return __uint_as_float(u);
#else
        float f;
        __builtin_memcpy(&f, &u, 4);
        return f;
#endif
    }
};

template <> struct KeyOf<double> {
    typedef unsigned long long type;
    static constexpr unsigned long long TOP = 0x8000000000000000ull;
    __host__ __device__ static inline unsigned long long enc(double f) {
#ifdef __CUDA_ARCH__
        unsigned long long u = (unsigned long long)__double_as_longlong(f);
#else
        unsigned long long u;
        __builtin_memcpy(&u, &f, 8);
#endif
        return (u & TOP) ? ~u : (u | TOP);
    }
    __host__ __device__ static inline double dec(unsigned long long k) {
        unsigned long long u = (k & TOP) ? (k & ~TOP) : ~k;
#ifdef __CUDA_ARCH__
        return __longlong_as_double((long long)u);
#else
        double f;
        __builtin_memcpy(&f, &u, 8);
        return f;
#endif
    }
};

// The keys of FP64 values are selected as they are (the FP64 tiles keep their
// maxima as keys, so that every comparison is an integer compare rather than an
// FP64 one): a key is its own key.
template <> struct KeyOf<unsigned long long> {
    typedef unsigned long long type;
    __host__ __device__ static inline unsigned long long enc(unsigned long long k) { return k; }
    __host__ __device__ static inline unsigned long long dec(unsigned long long k) { return k; }
};

}  // namespace pastila
