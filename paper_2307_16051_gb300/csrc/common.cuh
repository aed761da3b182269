// common.cuh — shared device/host helpers for the sm_103a kernels.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

namespace nl {

// ---------------------------------------------------------------- host side --

// Thread-local last-error text, surfaced by nl_last_error().
void set_error(const char* fmt, ...);
const char* get_error();

#define NL_CUDA_OK(expr)                                                                   \
    do {                                                                                   \
        cudaError_t _e = (expr);                                                           \
        if (_e != cudaSuccess) {                                                           \
            ::nl::set_error("%s:%d %s: %s", __FILE__, __LINE__, #expr, cudaGetErrorString(_e)); \
            return NL_ECUDA;                                                               \
        }                                                                                  \
    } while (0)

#define NL_TRY(expr)                    \
    do {                                \
        nl_status _s = (expr);          \
        if (_s != NL_OK) return _s;     \
    } while (0)

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }
inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

int num_sms();

// cudaMalloc for the handles' device pools; fails on purpose while the test
// hook nl_debug_fail_allocs has allocations left to fail.
cudaError_t dev_malloc(void** p, size_t bytes);

// Carves 256-byte aligned sub-buffers out of one device allocation (a null
// base only measures: off is the size needed).
struct Carver {
    char* base;
    size_t off = 0;
    explicit Carver(void* b) : base((char*)b) {}
    template <typename T>
    T* take(size_t n)
    {
        off = (off + 255) & ~(size_t)255;
        T* p = (T*)(base + off);
        off += n * sizeof(T);
        return p;
    }
};

// Optional per-kernel-class timing (nl_kernel_timing): when enabled for a
// class, every launch of it is bracketed by CUDA events on its stream.
void prof_begin(const char* kernel_class, cudaStream_t st);
void prof_end(const char* kernel_class, cudaStream_t st);

// Raise a kernel's dynamic shared-memory limit to the device's opt-in maximum
// minus the kernel's static shared memory.  Clears the runtime error state on
// failure and reports it as NL_ECUDA.
int set_max_dynamic_smem(const void* func);

// Device-side error word bits (solver status block).
enum : unsigned {
    ERR_TIMEOUT_TRSV = 1u << 0,  // a triangular-solve block gave up waiting on a predecessor
    ERR_TIMEOUT_OTHER = 1u << 1,
    ERR_NONFINITE = 1u << 2,
};

// Bounded spin limit for inter-CTA waits: about a second at the spin period.
constexpr long long kSpinLimit = 1LL << 24;

// -------------------------------------------------------------- device side --

__device__ __forceinline__ float round_h(float v) { return __half2float(__float2half_rn(v)); }

// fl16(fl32(a / b)) for a binary16 value b != 0 (held in a float) and
// rb = __frcp_rn(b), with no division and no branch.
//   q = fl32(a rb) is within 2^-22.9 |a/b| of a/b, hence so is fl32(a/b).
//   h = fl16(q).  Let m be the binary16 rounding boundary (the midpoint of
//   two adjacent binary16 values lo < hi) next to q on the side of q away
//   from h.  If |q - m| > 2^-21 |q|, no boundary separates q from fl32(a/b)
//   and h is the answer.  Otherwise the answer is decided exactly:
//   e = |a| - m |b| is exact (m |b| has at most 23 significant bits, and
//   Sterbenz's lemma applies), and fl32(|a/b|) > m iff e > up |b| / 2,
//   < m iff e < -dn |b| / 2 (up, dn: the single-precision spacings above and
//   below m; m has a zero last bit, so single-precision ties go to m), and
//   = m otherwise, when binary16 rounding of the tie picks the even one of
//   lo and hi.  The sign is that of q.  NaN and infinity follow q.
__device__ __forceinline__ float div_round_h(float a, float b, float rb)
{
    const float q = __fmul_rn(a, rb);
    const __half h = __float2half_rn(q);
    const float aq = fabsf(q);
    const unsigned hb = __half_as_ushort(h) & 0x7fffu;
    const float ah = __half2float(__ushort_as_half((unsigned short)hb));
    const unsigned nb = (aq > ah) ? hb + 1u : (hb ? hb - 1u : 0u);
    const float nf = __half2float(__ushort_as_half((unsigned short)nb));
    const float m = 0.5f * (ah + nf);
    const bool near = (aq != 0.0f) && (fabsf(aq - m) <= aq * 0x1p-21f);
    const float ab = fabsf(b);
    const float e = __fmaf_rn(-m, ab, fabsf(a));
    const unsigned mu = __float_as_uint(m);
    const float up = __fsub_rn(__uint_as_float(mu + 1u), m);
    const float dn = __fsub_rn(m, __uint_as_float(mu - 1u));
    const float sup = 0.5f * up * ab, sdn = 0.5f * dn * ab;
    const unsigned lob = min(hb, nb);
    const float lo = fminf(ah, nf), hi = fmaxf(ah, nf);
    const float exact = (e > sup) ? hi : ((-e > sdn) ? lo : ((lob & 1u) ? hi : lo));
    return copysignf(near ? exact : ah, q);
}

// The common case of div_round_h alone: fl16(fl32(a rb)), and in *unsure
// whether a binary16 rounding boundary lies within 2^-20 |q| of q (then the
// caller must use div_round_h; when *unsure is false the result is exact, by
// the same argument).
__device__ __forceinline__ float div_round_h_fast(float a, float rb, bool* unsure)
{
    const float q = __fmul_rn(a, rb);
    const __half h = __float2half_rn(q);
    const __half lo = __float2half_rn(__fmul_rn(q, 1.0f - 0x1p-20f));
    const __half hi = __float2half_rn(__fmul_rn(q, 1.0f + 0x1p-20f));
    *unsure = !(__half_as_ushort(lo) == __half_as_ushort(hi) && __half_as_ushort(h) == __half_as_ushort(lo));
    return __half2float(h);
}

// The sum of part[0 .. n) in index order, by every thread of the block (the
// last block of a grid-wide reduction): the partials are staged through
// shared memory a block's width at a time (parallel loads from L2) and thread
// 0 adds them in order, so the result is that of one thread's sequential
// loop; valid in thread 0.
__device__ __forceinline__ double ordered_sum_staged(const double* part, int n, double* buf)
{
    double t = 0.0;
    for (int base = 0; base < n; base += blockDim.x) {
        const int q = base + threadIdx.x;
        if (q < n) buf[threadIdx.x] = __ldcg(part + q);
        __syncthreads();
        if (threadIdx.x == 0) {
            const int m = min((int)blockDim.x, n - base);
            for (int e = 0; e < m; ++e) t += buf[e];
        }
        __syncthreads();
    }
    return t;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block-wide sum (fixed reduction tree).  `red` needs
// blockDim.x/32 entries.  Result valid in every thread.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    T s = T(0);
    for (int w = 0; w < nw; ++w) s += red[w];
    return s;
}

__device__ __forceinline__ int ld_acquire_gpu(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(int* p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Element loads/stores for the three factor storage types.
__device__ __forceinline__ float ld_elem(const __half* p) { return __half2float(*p); }
__device__ __forceinline__ float ld_elem(const float* p) { return *p; }
__device__ __forceinline__ double ld_elem(const double* p) { return *p; }
__device__ __forceinline__ void st_elem(__half* p, float v) { *p = __float2half_rn(v); }
__device__ __forceinline__ void st_elem(float* p, float v) { *p = v; }
__device__ __forceinline__ void st_elem(double* p, double v) { *p = v; }

}  // namespace nl
