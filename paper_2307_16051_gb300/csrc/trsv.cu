// trsv.cu — z = U^{-1} L^{-1} P v with the factors of the LU (Algorithm IR's
// correction d = U^{-1} L^{-1} r, Section 2.2; the preconditioner-vector
// product of GMRES-IR).  For the half-precision factors the binary16 entries
// are promoted to single as they are loaded and all arithmetic is single
// (interprecision transfer on the fly, eq. (2.16), Section 2.3).
//
// Blocked substitution with block size T.  The inverses of the T x T
// diagonal blocks of L and U are formed once per factorisation (in the
// solve precision), so each block step is a small matrix-vector product.
// One cooperative launch per triangle: CTA g owns block rows g, g+G, ...;
// a block row accumulates the contributions of the finished blocks as their
// readiness flags appear (epoch-tagged, acquire/release), then multiplies by
// the diagonal inverse and publishes its slice.  Every wait is bounded: after
// about a second the CTA records a timeout in the error word and all CTAs
// return, leaving the context usable.
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace nl {

constexpr int T_ = kTrsvT;
constexpr int kTrsvThreads = 256;           // 64 rows x 4 column quarters
constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at 2 GHz

template <typename T>
__device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }

// ---------------------------------------------------------------- prepare --

// Inverses of the diagonal blocks: Linv (unit lower) and Uinv (upper).
template <typename S, typename T>
__global__ void __launch_bounds__(T_) k_invdiag(int N, const S* __restrict__ LU, int64_t ld, T* __restrict__ dinv,
                                                int nblk)
{
    __shared__ T A[T_][T_ + 1];
    __shared__ T X[T_][T_ + 1];
    const int b = blockIdx.x, r0 = b * T_, nb_ = min(T_, N - r0);
    const int col = threadIdx.x;
    for (int i = 0; i < T_; ++i) A[i][col] = (i < nb_ && col < nb_) ? (T)ld_elem(LU + (int64_t)(r0 + i) * ld + r0 + col) : T(0);
    __syncthreads();
    // L^{-1} e_col by forward substitution (unit diagonal)
    for (int i = 0; i < T_; ++i) {
        T x = T(0);
        if (col < nb_ && i < nb_) {
            if (i == col) x = T(1);
            else if (i > col) {
                T s = T(0);
                for (int t = col; t < i; ++t) s = fma(A[i][t], X[t][col], s);
                x = -s;
            }
        }
        X[i][col] = x;
    }
    T* Linv = dinv + (int64_t)b * T_ * T_;
    for (int i = 0; i < T_; ++i) Linv[i * T_ + col] = X[i][col];
    // U^{-1} e_col by back substitution
    for (int i = T_ - 1; i >= 0; --i) {
        T x = T(0);
        if (col < nb_ && i < nb_ && i <= col) {
            T s = (i == col) ? T(1) : T(0);
            for (int t = i + 1; t <= col; ++t) s = fma(-A[i][t], X[t][col], s);
            x = s / A[i][i];
        }
        X[i][col] = x;
    }
    T* Uinv = dinv + (int64_t)(nblk + b) * T_ * T_;
    for (int i = 0; i < T_; ++i) Uinv[i * T_ + col] = X[i][col];
}

// Final row permutation from the LAPACK-style interchanges:
// perm[i] = original index of the entry that ends up at position i.
__global__ void __launch_bounds__(1024) k_perm(int N, const int* __restrict__ ipiv, int* __restrict__ perm,
                                               int* __restrict__ list)
{
    extern __shared__ int ps[];
    __shared__ int cnt[1024];
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < N; i += nt) ps[i] = i;
    // compact the non-trivial interchanges, keeping their order
    const int seg = (N + nt - 1) / nt, a = tid * seg, e = min(N, a + seg);
    int c = 0;
    for (int k = a; k < e; ++k) c += (ipiv[k] != k);
    cnt[tid] = c;
    __syncthreads();
    if (tid == 0) {
        int s = 0;
        for (int q = 0; q < nt; ++q) {
            int v = cnt[q];
            cnt[q] = s;
            s += v;
        }
        list[N] = s;
    }
    __syncthreads();
    int o = cnt[tid];
    for (int k = a; k < e; ++k)
        if (ipiv[k] != k) list[o++] = k;
    __syncthreads();
    if (tid == 0) {
        const int m = list[N];
        for (int q = 0; q < m; ++q) {
            int k = list[q], p = ipiv[k];
            int t = ps[k];
            ps[k] = ps[p];
            ps[p] = t;
        }
    }
    __syncthreads();
    for (int i = tid; i < N; i += nt) perm[i] = ps[i];
}

// ------------------------------------------------------------------ solve --

__device__ __forceinline__ bool wait_flag(const int* flag, int epoch, unsigned* err)
{
    long long t0 = clock64();
    while (ld_acquire_gpu(flag) != epoch) {
        if (*((volatile unsigned*)err) != 0u) return false;
        if (clock64() - t0 > kWaitCycles) {
            atomicOr(err, (unsigned)ERR_TIMEOUT_TRSV);
            return false;
        }
        __nanosleep(20);
    }
    return true;
}

// LOWER: forward solve y = L^{-1} P v (block rows in increasing order).
// !LOWER: back solve z = U^{-1} y (block rows in decreasing order).
template <typename S, typename T, bool LOWER>
__global__ void __launch_bounds__(kTrsvThreads) k_trsv(int N, int nblk, const S* __restrict__ LU, int64_t ld,
                                                      const T* __restrict__ v, const int* __restrict__ perm,
                                                      const T* __restrict__ dinv, T* __restrict__ out,
                                                      int* __restrict__ flags, int epoch, unsigned* __restrict__ err)
{
    __shared__ T xs[T_];
    __shared__ T acc[T_];
    __shared__ int abort_s;
    const int tid = threadIdx.x, r = tid >> 2, qq = tid & 3;
    const T* Dinv = dinv + (LOWER ? 0 : (int64_t)nblk * T_ * T_);
    for (int g = blockIdx.x; g < nblk; g += gridDim.x) {
        const int b = LOWER ? g : nblk - 1 - g;
        const int r0 = b * T_, row = r0 + r;
        if (tid < T_) {
            int i = r0 + tid;
            T x = T(0);
            if (i < N) x = LOWER ? v[perm[i]] : ldcg(v + i);
            acc[tid] = x;
        }
        T part = T(0);
        const S* Lrow = LU + (int64_t)min(row, N - 1) * ld;
        const int c_begin = LOWER ? 0 : nblk - 1, c_end = LOWER ? b : b, c_step = LOWER ? 1 : -1;
        for (int c = c_begin; c != c_end; c += c_step) {
            if (tid == 0) abort_s = wait_flag(flags + c, epoch, err) ? 0 : 1;
            __syncthreads();
            if (abort_s) return;
            if (tid < T_) {
                int i = c * T_ + tid;
                xs[tid] = (i < N) ? ldcg(out + i) : T(0);
            }
            __syncthreads();
            if (row < N) {
                const int cb = c * T_ + qq * 16;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    int col = cb + k;
                    T a = (col < N) ? (T)ld_elem(Lrow + col) : T(0);
                    part = fma(a, xs[qq * 16 + k], part);
                }
            }
        }
        part += __shfl_xor_sync(0xffffffffu, part, 1);
        part += __shfl_xor_sync(0xffffffffu, part, 2);
        __syncthreads();
        if (qq == 0) acc[r] -= part;
        __syncthreads();
        // slice = Dinv_b * acc
        const T* D = Dinv + (int64_t)b * T_ * T_ + r * T_ + qq * 16;
        T s = T(0);
#pragma unroll
        for (int k = 0; k < 16; ++k) s = fma(D[k], acc[qq * 16 + k], s);
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        if (qq == 0 && row < N) {
            out[row] = s;
            __threadfence();
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            st_release_gpu(flags + b, epoch);
        }
    }
}

// ------------------------------------------------------------------- host --

size_t trsv_work_bytes(int N, bool fp64)
{
    int nblk = (int)cdiv(N, T_);
    size_t el = fp64 ? 8 : 4;
    return round_up((size_t)N * 4, 256) + round_up((size_t)2 * nblk * T_ * T_ * el, 256) +
           round_up((size_t)2 * nblk * 4, 256) + round_up((size_t)N * el, 256) + 256 + round_up((size_t)(N + 1) * 4, 256);
}

void trsv_work_carve(void* base, int N, bool fp64, TrsvWork* w)
{
    int nblk = (int)cdiv(N, T_);
    size_t el = fp64 ? 8 : 4;
    char* p = (char*)base;
    w->perm = (int*)p;
    p += round_up((size_t)N * 4, 256);
    w->dinv = p;
    p += round_up((size_t)2 * nblk * T_ * T_ * el, 256);
    w->flags = (int*)p;
    p += round_up((size_t)2 * nblk * 4, 256);
    w->y = p;
    p += round_up((size_t)N * el, 256);
    w->err = (unsigned*)p;
    p += 256;
    w->scan = (int*)p;
}

template <typename S, typename T>
static nl_status prepare_impl(int N, const S* LU, int64_t ld, const int* ipiv, const TrsvWork& w, cudaStream_t st,
                              int* launches)
{
    const int nblk = (int)cdiv(N, T_);
    static bool attr = false;
    if (!attr) {
        NL_CUDA_OK(cudaFuncSetAttribute(k_perm, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        attr = true;
    }
    if ((size_t)N * 4 > 227 * 1024) {
        set_error("trsv: N=%d too large for the permutation kernel", N);
        return NL_EINVAL;
    }
    k_perm<<<1, 1024, (size_t)N * 4, st>>>(N, ipiv, w.perm, w.scan);
    k_invdiag<S, T><<<nblk, T_, 0, st>>>(N, LU, ld, (T*)w.dinv, nblk);
    NL_CUDA_OK(cudaGetLastError());
    if (launches) *launches += 2;
    return NL_OK;
}

nl_status trsv_prepare16(int N, const __half* LU, int64_t ld, const int* ipiv, const TrsvWork& w, cudaStream_t st,
                         int* launches)
{
    return prepare_impl<__half, float>(N, LU, ld, ipiv, w, st, launches);
}

nl_status trsv_prepare64(int N, const double* LU, int64_t ld, const int* ipiv, const TrsvWork& w, cudaStream_t st,
                         int* launches)
{
    return prepare_impl<double, double>(N, LU, ld, ipiv, w, st, launches);
}

template <typename S, typename T, bool LOWER>
static nl_status launch_trsv(int N, const S* LU, int64_t ld, const T* v, T* out, const TrsvWork& w, int epoch,
                             int* flags, cudaStream_t st)
{
    const int nblk = (int)cdiv(N, T_);
    auto kern = k_trsv<S, T, LOWER>;
    static int max_grid = 0;
    if (max_grid == 0) {
        int per_sm = 0;
        NL_CUDA_OK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTrsvThreads, 0));
        max_grid = std::max(1, per_sm) * num_sms();
    }
    int grid = std::min(nblk, max_grid);
    const int* perm = w.perm;
    const T* dinv = (const T*)w.dinv;
    unsigned* err = w.err;
    void* args[] = {(void*)&N, (void*)&nblk, (void*)&LU, (void*)&ld, (void*)&v, (void*)&perm, (void*)&dinv,
                    (void*)&out, (void*)&flags, (void*)&epoch, (void*)&err};
    NL_CUDA_OK(cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(kTrsvThreads), args, 0, st));
    return NL_OK;
}

template <typename S, typename T>
static nl_status solve_impl(int N, const S* LU, int64_t ld, const T* v, T* z, const TrsvWork& w, int epoch,
                            cudaStream_t st, int* launches)
{
    const int nblk = (int)cdiv(N, T_);
    T* y = (T*)w.y;
    nl_status s = launch_trsv<S, T, true>(N, LU, ld, v, y, w, epoch, w.flags, st);
    if (s != NL_OK) return s;
    s = launch_trsv<S, T, false>(N, LU, ld, y, z, w, epoch, w.flags + nblk, st);
    if (launches) *launches += 2;
    return s;
}

nl_status trsv_solve16(int N, const __half* LU, int64_t ld, const float* v, float* z, const TrsvWork& w, int epoch,
                       cudaStream_t st, int* launches)
{
    return solve_impl<__half, float>(N, LU, ld, v, z, w, epoch, st, launches);
}

nl_status trsv_solve64(int N, const double* LU, int64_t ld, const double* v, double* z, const TrsvWork& w, int epoch,
                       cudaStream_t st, int* launches)
{
    return solve_impl<double, double>(N, LU, ld, v, z, w, epoch, st, launches);
}

}  // namespace nl
