// Range-checked arrays and accesses for the bounds-check build.
//
// Compiled with -DMPPI_BOUNDS_CHECK, every index into the device
// workspaces, the staged model and the kernels' shared memory (CArr below)
// and every global-memory index at the kernels' access sites (MPPI_IN_RANGE)
// is compared with its extent.  A failed check sets a bit in this
// translation unit's bounds word and the access goes to a sink instead of
// the array: no trap, no fault.  mppi_debug_bounds() reads and clears the
// words of every translation unit.  Without the flag, CArr is a plain array
// and the checks compile to nothing.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace mppi {

// bits of the bounds word
constexpr unsigned BOUNDS_SHARED = 1u;  // an index into a workspace / shared array
constexpr unsigned BOUNDS_GLOBAL = 2u;  // an index into a caller's or handle's device buffer

#ifdef MPPI_BOUNDS_CHECK
constexpr bool kBoundsCheck = true;
// one word and one sink per translation unit (no relocatable device code)
static __device__ unsigned int g_bounds_word;
static __device__ __align__(16) unsigned char g_bounds_sink[2048];  // >= the largest row type
__device__ __forceinline__ void bounds_fail(unsigned bit) { atomicOr(&g_bounds_word, bit); }
#else
constexpr bool kBoundsCheck = false;
#endif

// A fixed-size array whose operator[] checks the index in the bounds-check
// build (device code only; the host fills the model with plain accesses).
// Same size, alignment and layout as T[N]; converts to T* so that a row can
// be handed on as a pointer.
template <class T, int N>
struct CArr {
    T v[N];
    __host__ __device__ __forceinline__ T& operator[](int i) {
#if defined(MPPI_BOUNDS_CHECK) && defined(__CUDA_ARCH__)
        if ((unsigned)i >= (unsigned)N) {
            bounds_fail(BOUNDS_SHARED);
            static_assert(sizeof(T) <= sizeof(g_bounds_sink), "sink smaller than the row type");
            return *reinterpret_cast<T*>(g_bounds_sink);
        }
#endif
        return v[i];
    }
    __host__ __device__ __forceinline__ const T& operator[](int i) const {
#if defined(MPPI_BOUNDS_CHECK) && defined(__CUDA_ARCH__)
        if ((unsigned)i >= (unsigned)N) {
            bounds_fail(BOUNDS_SHARED);
            return *reinterpret_cast<const T*>(g_bounds_sink);
        }
#endif
        return v[i];
    }
    __host__ __device__ __forceinline__ operator T*() { return v; }
    __host__ __device__ __forceinline__ operator const T*() const { return v; }
};

// True when 0 <= i < n; in the bounds-check build a false result also sets
// the global-buffer bit.  Use as `if (MPPI_IN_RANGE(i, n)) p[i] = ...` or
// around a read whose fallback keeps the lane's value.
__device__ __forceinline__ bool in_range_dev(long long i, long long n) {
#ifdef MPPI_BOUNDS_CHECK
    if (i < 0 || i >= n) {
        bounds_fail(BOUNDS_GLOBAL);
        return false;
    }
#endif
    (void)i;
    (void)n;
    return true;
}
#define MPPI_IN_RANGE(i, n) (::mppi::in_range_dev((long long)(i), (long long)(n)))

// A checked read of a global buffer: p[i] when 0 <= i < n, else 0 (and the
// bit set) in the bounds-check build.
template <class T>
__device__ __forceinline__ T ld_checked(const T* p, long long i, long long n) {
#ifdef MPPI_BOUNDS_CHECK
    if (i < 0 || i >= n) {
        bounds_fail(BOUNDS_GLOBAL);
        return T{};
    }
#endif
    (void)n;
    return p[i];
}

}  // namespace mppi

// Each translation unit with kernels defines its reader of the word with
// MPPI_BOUNDS_READER(name): unsigned name() returns and clears it (0 in the
// normal build).
#ifdef MPPI_BOUNDS_CHECK
#define MPPI_BOUNDS_READER(name)                                                             \
    unsigned name() {                                                                        \
        unsigned v = 0, z = 0;                                                               \
        if (cudaMemcpyFromSymbol(&v, ::mppi::g_bounds_word, sizeof v) != cudaSuccess) return ~0u; \
        cudaMemcpyToSymbol(::mppi::g_bounds_word, &z, sizeof z);                             \
        return v;                                                                            \
    }
#else
#define MPPI_BOUNDS_READER(name) \
    unsigned name() { return 0u; }
#endif
