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

namespace cg = cooperative_groups;

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

// ---------------------------------------------- single-precision mailbox --
// For the single-precision solve each solved entry is published as one 64-bit
// word {value bits, epoch} with a release store; a consumer polls the word of
// the entry it needs with an acquire load, so readiness and data arrive
// together in one memory round trip.  Block size 128: the diagonal inverse
// (64 KB) is staged in shared memory and each thread prefetches its 64
// binary16 entries of the next tile before polling.
constexpr int T2 = 128;
constexpr int kMbThreads = 256;  // 128 rows x 2 halves of 64 columns

// A published word carries its own readiness (the epoch) and its value, and a
// consumer reads nothing else the producer wrote, so relaxed GPU-scope accesses
// suffice (no acquire / release, hence no cache invalidation per poll).
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Bounded poll of one published entry: false once `limit` cycles have passed
// (a negative limit gives up before the first poll: the test of the timeout
// path, a wait that runs out whatever the producer does).
__device__ __forceinline__ bool poll_value(const unsigned long long* p, unsigned epoch, float* out,
                                           const unsigned* err, long long limit)
{
    if (limit < 0) return false;
    long long t0 = clock64();
    for (;;) {
        unsigned long long w = ld_relaxed_u64(p);
        if ((unsigned)(w >> 32) == epoch) {
            *out = __uint_as_float((unsigned)w);
            return true;
        }
        if (*((volatile const unsigned*)err) != 0u) return false;
        if (clock64() - t0 > limit) return false;
    }
}

template <bool LOWER>
__global__ void __launch_bounds__(kMbThreads) k_trsv_mb(int N, int nblk, const __half* __restrict__ LU, int64_t ld,
                                                       const float* __restrict__ v,
                                                       const unsigned long long* __restrict__ vin_mb,
                                                       const int* __restrict__ perm, const float* __restrict__ dinv,
                                                       unsigned long long* __restrict__ mb, float* __restrict__ out,
                                                       unsigned epoch, unsigned* __restrict__ err, long long wait_cycles,
                                                       const float* __restrict__ rs)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* Ds = reinterpret_cast<float*>(smem_raw);  // T2 x T2 diagonal inverse
    __shared__ float ys[T2];
    __shared__ float acc[T2];
    const int tid = threadIdx.x, r = tid >> 1, h = tid & 1;
    const float* Dinv = dinv + (LOWER ? 0 : (int64_t)nblk * T2 * T2);
    for (int g = blockIdx.x; g < nblk; g += gridDim.x) {
        const int b = LOWER ? g : nblk - 1 - g;
        const int r0 = b * T2, row = r0 + r;
        // stage this block's diagonal inverse (independent of the waits)
        __syncthreads();
        {
            const float4* src = reinterpret_cast<const float4*>(Dinv + (int64_t)b * T2 * T2);
            float4* dst = reinterpret_cast<float4*>(Ds);
            for (int q = tid; q < T2 * T2 / 4; q += kMbThreads) dst[q] = src[q];
        }
        if (tid < T2) {
            const int i = r0 + tid;
            float x = 0.0f;
            if (i < N)
                x = LOWER ? (rs ? v[perm[i]] * rs[perm[i]] : v[perm[i]]) : __uint_as_float((unsigned)vin_mb[i]);
            acc[tid] = x;
        }
        float part = 0.0f;
        const __half* Lrow = LU + (int64_t)min(row, N - 1) * ld;
        const int cnt = LOWER ? b : nblk - 1 - b;
        // this thread's 64 entries of tile (b, c), loaded one tile ahead of their use
        auto fetch = [&](int c, __half2* dst) {
            const int cb = c * T2 + h * 64;
            if (row < N && cb + 64 <= N && (((uintptr_t)(Lrow + cb)) & 15) == 0) {
                const uint4* p4 = reinterpret_cast<const uint4*>(Lrow + cb);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    uint4 u = __ldcs(p4 + q);  // streamed once: do not keep it in the caches
                    memcpy(&dst[4 * q], &u, 16);
                }
            } else {
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    int c0 = cb + 2 * q;
                    float a0 = (row < N && c0 < N) ? __half2float(Lrow[c0]) : 0.0f;
                    float a1 = (row < N && c0 + 1 < N) ? __half2float(Lrow[c0 + 1]) : 0.0f;
                    dst[q] = __floats2half2_rn(a0, a1);
                }
            }
        };
        __half2 lv[32], nx[32];
        if (cnt > 0) fetch(LOWER ? 0 : nblk - 1, lv);
        for (int s = 0; s < cnt; ++s) {
            const int c = LOWER ? s : nblk - 1 - s;
            if (s + 1 < cnt) fetch(LOWER ? s + 1 : nblk - 2 - s, nx);
            __syncthreads();  // ys of the previous tile no longer in use
            bool okp = true;
            if (tid < T2) {
                const int i = c * T2 + tid;
                float y = 0.0f;
                if (i < N) okp = poll_value(mb + i, epoch, &y, err, wait_cycles);
                ys[tid] = y;
            }
            if (__syncthreads_or(!okp)) {
                if (tid == 0) atomicOr(err, (unsigned)ERR_TIMEOUT_TRSV);
                return;
            }
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                float2 f = __half22float2(lv[q]);
                part = fmaf(f.x, ys[h * 64 + 2 * q], part);
                part = fmaf(f.y, ys[h * 64 + 2 * q + 1], part);
            }
#pragma unroll
            for (int q = 0; q < 32; ++q) lv[q] = nx[q];
        }
        part += __shfl_xor_sync(0xffffffffu, part, 1);
        __syncthreads();
        if (h == 0) acc[r] -= part;
        __syncthreads();
        float sum = 0.0f;
#pragma unroll 16
        for (int k = 0; k < 64; ++k) sum = fmaf(Ds[r * T2 + h * 64 + k], acc[h * 64 + k], sum);
        sum += __shfl_xor_sync(0xffffffffu, sum, 1);
        if (h == 0 && row < N) {
            if (out) out[row] = sum;
            st_relaxed_u64(mb + row, ((unsigned long long)epoch << 32) | __float_as_uint(sum));
        }
    }
}

// ------------------------------------------------ cluster triangular solve --
// One thread-block cluster of C CTAs (C <= 16) solves the whole triangle.
// Block b of 128 rows belongs to CTA (step of b) mod C, which keeps the
// running right-hand side of its blocks in shared memory.  The owner of step
// s forms z_b = Dinv_b acc_b and stores z_b into every CTA's shared memory
// with st.async, each store completing a transaction count on that CTA's
// mbarrier for step s (one mbarrier per block, used once).  A CTA waits
// only for the z it needs next; the owner of step s+1 first subtracts
// L(b(s+1), b(s)) z_s, with the tile already in registers, then publishes
// z_{b(s+1)} before it applies z_s to its other blocks, so the chain from
// one block to the next is one shared-memory signal, one 128 x 32 update
// per thread group and one 128 x 128 product with the inverse (also held
// in registers).  Every row of the factor is read by exactly one CTA.
// Shared vectors of 128 floats are padded to 132 (column c at c + c/32) so
// the four column quarters fall in different banks.
constexpr int kClThreads = 512;  // 128 rows x 4 column quarters of 32
constexpr int kClPad = 132;
constexpr int kClMaxSmem = 220 * 1024;
constexpr long long kClWaitIters = 1LL << 24;

// Dynamic shared memory: nblk mbarriers, then nblk + nown padded vectors.
__host__ __device__ inline int trsv_cl_bar_bytes(int nblk) { return (nblk * 8 + 15) & ~15; }
inline size_t trsv_cl_smem(int nblk, int nown)
{
    return (size_t)trsv_cl_bar_bytes(nblk) + (size_t)(nblk + nown) * kClPad * sizeof(float);
}

__device__ __forceinline__ uint32_t cl_smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint32_t cl_mapa(uint32_t a, int rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void cl_st_async(uint32_t addr, float v, uint32_t bar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(addr),
                 "r"(__float_as_uint(v)), "r"(bar)
                 : "memory");
}
// Bounded wait for phase 0 of a local mbarrier; false after `iters` polls
// (kClWaitIters by default; 0 gives up at once, the test of the timeout path).
__device__ __forceinline__ bool cl_wait(uint32_t bar, long long iters = kClWaitIters)
{
    for (long long it = 0; it < iters; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], 0;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Row i of the factor, columns c0 .. c0+31 (zeros outside the matrix).
__device__ __forceinline__ void cl_load_tile(const __half* __restrict__ LU, int64_t ld, int N, int i, int c0,
                                             bool vecld, uint4 (&t)[4])
{
    if (i < N && vecld && c0 + 32 <= N) {
        const uint4* p = reinterpret_cast<const uint4*>(LU + (int64_t)i * ld + c0);
#pragma unroll
        for (int q = 0; q < 4; ++q) t[q] = p[q];
    } else {
        __half h[32];
#pragma unroll
        for (int k = 0; k < 32; ++k)
            h[k] = (i < N && c0 + k < N) ? LU[(int64_t)i * ld + c0 + k] : __float2half_rn(0.0f);
        memcpy(t, h, 64);
    }
}
__device__ __forceinline__ float cl_dot_tile(const uint4 (&t)[4], const float* __restrict__ z)
{
    float part = 0.0f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const __half2* h2 = reinterpret_cast<const __half2*>(&t[q]);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float2 f = __half22float2(h2[e]);
            part = fmaf(f.x, z[8 * q + 2 * e], part);
            part = fmaf(f.y, z[8 * q + 2 * e + 1], part);
        }
    }
    return part;
}

template <bool LOWER>
__global__ void __launch_bounds__(kClThreads, 1) k_trsv_cl(int N, int nblk, const __half* __restrict__ LU, int64_t ld,
                                                       const float* __restrict__ v, const int* __restrict__ perm,
                                                       const float* __restrict__ dinv, float* __restrict__ out,
                                                       unsigned* __restrict__ err, long long wait_iters,
                                                       const float* __restrict__ rs)
{
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    extern __shared__ __align__(16) unsigned char cl_raw[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(cl_raw);
    float* yv = reinterpret_cast<float*>(cl_raw + trsv_cl_bar_bytes(nblk));  // solved blocks, padded
    float* acc = yv + (size_t)nblk * kClPad;                                       // this CTA's blocks, padded
    __shared__ int abort_cta;
    const int tid = threadIdx.x, row = tid >> 2, qq = tid & 3;
    const int prow = row + (row >> 5);  // padded position of this row
    const float* Dinv = dinv + (LOWER ? 0 : (int64_t)nblk * T2 * T2);
    const int nown = (nblk - rank + C - 1) / C;
    const bool vecld = ((((uintptr_t)LU) & 15) == 0) && ((ld * 2) % 16 == 0);
    auto blk = [&](int s) { return LOWER ? s : nblk - 1 - s; };
    for (int j = 0; j < nown; ++j) {
        const int bj = blk(rank + j * C);
        for (int t = tid; t < T2; t += kClThreads) {
            const int i = bj * T2 + t;
            acc[j * kClPad + t + (t >> 5)] =
                (i < N) ? (LOWER ? (rs ? v[perm[i]] * rs[perm[i]] : v[perm[i]]) : v[i]) : 0.0f;
        }
    }
    if (tid == 0) {
        abort_cta = 0;
        for (int s = 0; s < nblk; ++s) {
            const uint32_t a = cl_smem_u32(bar + s);
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a));
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(T2 * 4) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    cl.sync();  // barriers initialised and every CTA running before the first remote store

    float4 dq[8];  // this thread's quarter of row `row` of the inverse of the next block it publishes
    uint4 ct[4];   // its 32 factor entries of the next tile on its chain
    auto load_D = [&](int b) {
        const float4* D = reinterpret_cast<const float4*>(Dinv + (int64_t)b * T2 * T2 + row * T2 + qq * 32);
#pragma unroll
        for (int k = 0; k < 8; ++k) dq[k] = D[k];
    };
    // z_b = Dinv_b acc_b for the step s this CTA owns, stored into every CTA
    auto publish = [&](int s) {
        const int b = blk(s);
        const float* a = acc + (s / C) * kClPad + qq * 33;
        float sum = 0.0f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            sum = fmaf(dq[k].x, a[4 * k], sum);
            sum = fmaf(dq[k].y, a[4 * k + 1], sum);
            sum = fmaf(dq[k].z, a[4 * k + 2], sum);
            sum = fmaf(dq[k].w, a[4 * k + 3], sum);
        }
        sum += __shfl_xor_sync(0xffffffffu, sum, 1);
        sum += __shfl_xor_sync(0xffffffffu, sum, 2);
        if (qq == 0) {
            const uint32_t ya = cl_smem_u32(yv + (size_t)b * kClPad + prow), ba = cl_smem_u32(bar + s);
            for (int c = 0; c < C; ++c) cl_st_async(cl_mapa(ya, c), sum, cl_mapa(ba, c));
            const int i = b * T2 + row;
            if (i < N) out[i] = sum;
        }
        if (s + C < nblk) {
            // inverse and chain tile for this CTA's next step s + C
            load_D(blk(s + C));
            cl_load_tile(LU, ld, N, blk(s + C) * T2 + row, blk(s + C - 1) * T2 + qq * 32, vecld, ct);
        }
    };
    if (rank < nblk) load_D(blk(rank));
    if (rank >= 1 && rank < nblk) cl_load_tile(LU, ld, N, blk(rank) * T2 + row, blk(rank - 1) * T2 + qq * 32, vecld, ct);
    if (rank == 0) publish(0);
    for (int s = 0; s < nblk; ++s) {
        const int b = blk(s);
        bool ok = false;
        if (!*((volatile int*)&abort_cta)) {
            ok = cl_wait(cl_smem_u32(bar + s), wait_iters);
            if (!ok) {
                abort_cta = 1;
                atomicOr(err, (unsigned)ERR_TIMEOUT_TRSV);
            }
        }
        const float* z = yv + (size_t)b * kClPad + qq * 33;
        int j = (s < rank) ? 0 : (s - rank) / C + 1;  // this CTA's blocks solved after step s
        if (j < nown && rank + j * C == s + 1) {
            // next block on the chain: update with the tile already in registers, then publish it
            const float part0 = ok ? cl_dot_tile(ct, z) : 0.0f;
            float part = part0 + __shfl_xor_sync(0xffffffffu, part0, 1);
            part += __shfl_xor_sync(0xffffffffu, part, 2);
            if (qq == 0) acc[j * kClPad + prow] -= part;
            __syncthreads();
            publish(s + 1);
            ++j;
        }
        if (!ok) continue;
        for (; j < nown; ++j) {
            uint4 t[4];
            cl_load_tile(LU, ld, N, blk(rank + j * C) * T2 + row, b * T2 + qq * 32, vecld, t);
            float part = cl_dot_tile(t, z);
            part += __shfl_xor_sync(0xffffffffu, part, 1);
            part += __shfl_xor_sync(0xffffffffu, part, 2);
            if (qq == 0) acc[j * kClPad + prow] -= part;
        }
    }
    // After a wait gave up, the owners of the later steps still publish them
    // (their values unused), so every mbarrier of this CTA still completes:
    // wait for all of them (the default bound) before leaving, so that no
    // st.async into this CTA's shared memory is still in flight when it exits.
    __syncthreads();
    if (*((volatile int*)&abort_cta))
        for (int s = 0; s < nblk; ++s) cl_wait(cl_smem_u32(bar + s));
    cl.sync();  // no CTA leaves before every CTA has passed all of its waits
}

// ------------------------------------------------------------------- host --

static int trsv_block(bool fp64) { return fp64 ? T_ : T2; }

size_t trsv_work_bytes(int N, bool fp64)
{
    const int tb = trsv_block(fp64);
    int nblk = (int)cdiv(N, tb);
    size_t el = fp64 ? 8 : 4;
    return round_up((size_t)N * 4, 256) + round_up((size_t)2 * nblk * tb * tb * el, 256) +
           round_up((size_t)2 * nblk * 4, 256) + round_up((size_t)N * 8 * 2, 256) + 256 +
           round_up((size_t)(N + 1) * 4, 256);
}

void trsv_work_carve(void* base, int N, bool fp64, TrsvWork* w)
{
    const int tb = trsv_block(fp64);
    int nblk = (int)cdiv(N, tb);
    size_t el = fp64 ? 8 : 4;
    char* p = (char*)base;
    w->perm = (int*)p;
    p += round_up((size_t)N * 4, 256);
    w->dinv = p;
    p += round_up((size_t)2 * nblk * tb * tb * el, 256);
    w->flags = (int*)p;
    p += round_up((size_t)2 * nblk * 4, 256);
    w->y = p;  // double: N elements; float: 2 x N 64-bit mailbox words
    p += round_up((size_t)N * 8 * 2, 256);
    w->err = (unsigned*)p;
    p += 256;
    w->scan = (int*)p;
}

// Diagonal-block inverses for block size TB, one thread per column, both
// right-looking: once X's row t of the column is final, it is applied to every
// later row, so the loop over rows has no dependence chain.  L (unit lower):
// entry i of column c is -sum_{t=c}^{i-1} l_it x_t with the terms added in
// increasing t, x_c = 1.  U: x_t = s_t / u_tt with s_i = [i == c] -
// sum_{t>i} u_it x_t, the terms added in decreasing t.  Entries outside the
// block (a ragged last block) are zero.
// x[i] <- fma(a[i], y, x[i]) for rows i in [i0, i1) of one column (stride TB + 1);
// rows in groups of four so the shared-memory loads run ahead of the stores.
// fma(a, -y, x) is the same operation as fma(-a, y, x).
template <typename T, int TB>
__device__ __forceinline__ void axpy_col(const T* __restrict__ a, T* __restrict__ x, int i0, int i1, T y)
{
    constexpr int S = TB + 1;
    int i = i0;
    for (; i + 4 <= i1; i += 4) {
        const T a0 = a[i * S], a1 = a[(i + 1) * S], a2 = a[(i + 2) * S], a3 = a[(i + 3) * S];
        const T x0 = x[i * S], x1 = x[(i + 1) * S], x2 = x[(i + 2) * S], x3 = x[(i + 3) * S];
        x[i * S] = fma(a0, y, x0);
        x[(i + 1) * S] = fma(a1, y, x1);
        x[(i + 2) * S] = fma(a2, y, x2);
        x[(i + 3) * S] = fma(a3, y, x3);
    }
    for (; i < i1; ++i) x[i * S] = fma(a[i * S], y, x[i * S]);
}

template <typename S, typename T, int TB>
__global__ void __launch_bounds__(TB) k_invdiag_t(int N, const S* __restrict__ LU, int64_t ld, T* __restrict__ dinv,
                                                  int nblk)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* A = reinterpret_cast<T*>(smem_raw);  // TB x (TB+1)
    T* X = A + TB * (TB + 1);
    const int b = blockIdx.x, r0 = b * TB, nb_ = min(TB, N - r0);
    const int col = threadIdx.x;
    T* x = X + col;  // this thread's column: x[i * (TB + 1)]
    for (int i = 0; i < TB; ++i)
        A[i * (TB + 1) + col] = (i < nb_ && col < nb_) ? (T)ld_elem(LU + (int64_t)(r0 + i) * ld + r0 + col) : T(0);
    for (int i = 0; i < TB; ++i) x[i * (TB + 1)] = T(0);
    __syncthreads();
    // L^{-1}
    for (int t = 0; t < nb_; ++t) {
        if (t < col || col >= nb_) continue;
        const T xt = (t == col) ? T(1) : -x[t * (TB + 1)];
        x[t * (TB + 1)] = xt;
        axpy_col<T, TB>(A + t, x, t + 1, nb_, xt);
    }
    T* Linv = dinv + (int64_t)b * TB * TB;
    for (int i = 0; i < TB; ++i) Linv[i * TB + col] = x[i * (TB + 1)];
    // U^{-1}
    for (int i = 0; i < TB; ++i) x[i * (TB + 1)] = (i == col && col < nb_) ? T(1) : T(0);
    for (int t = nb_ - 1; t >= 0; --t) {
        if (t > col || col >= nb_) continue;
        const T xt = x[t * (TB + 1)] / A[t * (TB + 1) + t];
        x[t * (TB + 1)] = xt;
        axpy_col<T, TB>(A + t, x, 0, t, -xt);
    }
    T* Uinv = dinv + (int64_t)(nblk + b) * TB * TB;
    for (int i = 0; i < TB; ++i) Uinv[i * TB + col] = x[i * (TB + 1)];
}

// The binary16 factors' 128 x 128 diagonal-block inverses, the same
// right-looking recurrences as k_invdiag_t with the column in registers:
// four threads per column (lane = 4 x column-in-warp + quarter), thread q
// holding rows 32q..32q+31.  At step t the thread holding row t finalises it
// and passes x_t to the column's other three threads with one shuffle; every
// thread then applies x_t to all 32 of its rows with the block's column t
// (staged transposed in shared memory with the entries the step must not
// touch — on and above the diagonal for L, on and below it for U — set to
// zero, so the update needs no per-row test and leaves them unchanged).
constexpr int kInvThreads = 512;
constexpr int kInvS = 148;  // transposed column stride (floats): quarters 36 apart; 148 t mod 32 spreads the staging stores
constexpr size_t kInvSmem = (size_t)T2 * kInvS * sizeof(float) + T2 * sizeof(float);

template <bool UPPER>
__device__ __forceinline__ void invdiag16_pass(const __half* __restrict__ LU, int64_t ld, float* __restrict__ D, int r0,
                                               int nb_)
{
    extern __shared__ __align__(16) float inv_sm[];
    float* At = inv_sm;             // At[t * kInvS + 36 q + r]: entry (32 q + r, t)
    float* dg = inv_sm + T2 * kInvS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int col = warp * 8 + (lane >> 2), q = lane & 3;
    for (int e = tid; e < T2 * T2; e += kInvThreads) {
        const int i = e / T2, t = e % T2;  // row i, column t of the block
        float a = 0.0f;
        if (i < nb_ && t < nb_) {
            const float v = __half2float(LU[(int64_t)(r0 + i) * ld + r0 + t]);
            if (UPPER ? (i < t) : (i > t)) a = UPPER ? -v : v;
            if (i == t) dg[t] = v;
        }
        At[t * kInvS + 36 * (i >> 5) + (i & 31)] = a;
    }
    __syncthreads();
    float acc[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) acc[r] = (UPPER && 32 * q + r == col && col < nb_) ? 1.0f : 0.0f;
    for (int s = 0; s < T2 / 32; ++s) {
        const int tq = UPPER ? 3 - s : s;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const int tt = UPPER ? 31 - k : k;
            const int t = 32 * tq + tt;
            float xt = 0.0f;
            if (q == tq && col < nb_ && t < nb_) {
                if (UPPER)
                    xt = (t > col) ? 0.0f : acc[tt] / dg[t];
                else
                    xt = (t < col) ? 0.0f : ((t == col) ? 1.0f : -acc[tt]);
                acc[tt] = xt;
            }
            xt = __shfl_sync(0xffffffffu, xt, (lane & ~3) | tq);
            const float4* a4 = reinterpret_cast<const float4*>(At + t * kInvS + 36 * q);
#pragma unroll
            for (int g = 0; g < 8; ++g) {
                const float4 v = a4[g];
                acc[4 * g] = fmaf(v.x, xt, acc[4 * g]);
                acc[4 * g + 1] = fmaf(v.y, xt, acc[4 * g + 1]);
                acc[4 * g + 2] = fmaf(v.z, xt, acc[4 * g + 2]);
                acc[4 * g + 3] = fmaf(v.w, xt, acc[4 * g + 3]);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 32; ++r) D[(32 * q + r) * T2 + col] = acc[r];
}

// CTA b < nblk: L^{-1} of block b; CTA nblk + b: U^{-1} of block b (U's
// entries are staged negated, so both updates are fma(a, x_t, acc)).
__global__ void __launch_bounds__(kInvThreads) k_invdiag16(int N, const __half* __restrict__ LU, int64_t ld,
                                                           float* __restrict__ dinv, int nblk)
{
    const bool upper = (int)blockIdx.x >= nblk;
    const int b = upper ? (int)blockIdx.x - nblk : (int)blockIdx.x;
    const int r0 = b * T2, nb_ = min(T2, N - r0);
    float* D = dinv + (int64_t)blockIdx.x * T2 * T2;
    if (upper)
        invdiag16_pass<true>(LU, ld, D, r0, nb_);
    else
        invdiag16_pass<false>(LU, ld, D, r0, nb_);
}

template <typename S, typename T>
static nl_status prepare_impl(int N, const S* LU, int64_t ld, const int* ipiv, const TrsvWork& w, cudaStream_t st,
                              int* launches)
{
    constexpr bool fp64 = std::is_same<T, double>::value;
    constexpr int TB = std::is_same<S, __half>::value ? T2 : T_;  // the block size of the solve that follows
    const int nblk = (int)cdiv(N, TB);
    static bool attr = false;
    if (!attr) {
        if (set_max_dynamic_smem((const void*)k_perm) != NL_OK ||
            set_max_dynamic_smem((const void*)k_invdiag_t<S, T, TB>) != NL_OK ||
            set_max_dynamic_smem((const void*)k_invdiag16) != NL_OK)
            return NL_ECUDA;
        attr = true;
    }
    if ((size_t)N * 4 > 200 * 1024) {
        set_error("trsv: N=%d too large for the permutation kernel", N);
        return NL_EINVAL;
    }
    k_perm<<<1, 1024, (size_t)N * 4, st>>>(N, ipiv, w.perm, w.scan);
    prof_begin("k_invdiag", st);
    if constexpr (std::is_same<S, __half>::value && !fp64)
        k_invdiag16<<<2 * nblk, kInvThreads, kInvSmem, st>>>(N, LU, ld, (float*)w.dinv, nblk);
    else
        k_invdiag_t<S, T, TB><<<nblk, TB, (size_t)2 * TB * (TB + 1) * sizeof(T), st>>>(N, LU, ld, (T*)w.dinv, nblk);
    prof_end("k_invdiag", st);
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

nl_status trsv_prepare32(int N, const float* LU, int64_t ld, const int* ipiv, const TrsvWork& w, cudaStream_t st,
                         int* launches)
{
    return prepare_impl<float, float>(N, LU, ld, ipiv, w, st, launches);
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

template <bool LOWER>
static nl_status launch_trsv_mb(int N, const __half* LU, int64_t ld, const float* v, const unsigned long long* vin_mb,
                                unsigned long long* mb, float* out, const TrsvWork& w, unsigned epoch, cudaStream_t st)
{
    const int nblk = (int)cdiv(N, T2);
    auto kern = k_trsv_mb<LOWER>;
    const size_t smem = (size_t)T2 * T2 * sizeof(float);
    static int max_grid = 0;
    if (max_grid == 0) {
        if (set_max_dynamic_smem((const void*)kern) != NL_OK) return NL_ECUDA;
        int per_sm = 0;
        NL_CUDA_OK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kMbThreads, smem));
        max_grid = std::max(1, per_sm) * num_sms();
    }
    int grid = std::min(nblk, max_grid);
    const int* perm = w.perm;
    const float* dinv = (const float*)w.dinv;
    unsigned* err = w.err;
    long long wait = w.wait_limit == 0 ? kWaitCycles : (w.wait_limit < 0 ? -1LL : (long long)w.wait_limit);
    const float* rs = w.rs;
    void* args[] = {(void*)&N,   (void*)&nblk, (void*)&LU,  (void*)&ld,    (void*)&v,   (void*)&vin_mb, (void*)&perm,
                    (void*)&dinv, (void*)&mb, (void*)&out, (void*)&epoch, (void*)&err, (void*)&wait, (void*)&rs};
    prof_begin("k_trsv_mb", st);
    cudaError_t le = cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(kMbThreads), args, smem, st);
    prof_end("k_trsv_mb", st);
    NL_CUDA_OK(le);
    return NL_OK;
}

// Whether a cluster of C CTAs of the cluster triangular solve can be
// co-scheduled on this device (cached per process; C in {4, 8, 16}).
static bool trsv_cluster_ok(int C)
{
    static int avail[3] = {-1, -1, -1};
    const int slot = C == 16 ? 2 : (C == 8 ? 1 : 0);
    if (avail[slot] < 0) {
        bool ok = true;
        for (int low = 0; low < 2 && ok; ++low) {
            const void* kern = low ? (const void*)k_trsv_cl<true> : (const void*)k_trsv_cl<false>;
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kClMaxSmem) != cudaSuccess) {
                ok = false;
                break;
            }
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = C;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(C);
            cfg.blockDim = dim3(kClThreads);
            cfg.dynamicSmemBytes = kClMaxSmem;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess || n < 1) ok = false;
        }
        cudaGetLastError();
        avail[slot] = ok ? 1 : 0;
    }
    return avail[slot] == 1;
}

// Cluster size for nblk blocks under the request req (0 = largest available,
// -1 = none, else the largest available <= req); 0 = use the mailbox solve.
// Automatic choice: the cluster's 16 SMs stream the whole factor, so beyond
// 80 blocks (N > 10240) the mailbox solve over all SMs is faster (measured on
// GB300: 197 vs 247 us at N = 8192, 379 vs 368 us at 12288, 676 vs 489 us at
// 16384 per triangle).
constexpr int kClAutoMaxBlocks = 80;
static int trsv_cluster_size(int nblk, int req)
{
    if (req < 0 || (req == 0 && nblk > kClAutoMaxBlocks)) return 0;
    for (int C : {16, 8, 4})
        if ((req == 0 || C <= req) && trsv_cluster_ok(C)) {
            const int Cn = std::min(C, nblk);
            if (trsv_cl_smem(nblk, (int)cdiv(nblk, Cn)) > (size_t)kClMaxSmem) return 0;
            return Cn;
        }
    return 0;
}

template <bool LOWER>
static nl_status launch_trsv_cl(int N, const __half* LU, int64_t ld, const float* v, float* out, const TrsvWork& w,
                                int C, cudaStream_t st)
{
    const int nblk = (int)cdiv(N, T2);
    const int nown = (int)cdiv(nblk, C);
    const size_t smem = trsv_cl_smem(nblk, nown);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int* perm = w.perm;
    const float* dinv = (const float*)w.dinv;
    prof_begin("k_trsv_cl", st);
    const long long wait = w.wait_limit == 0 ? kClWaitIters : (w.wait_limit < 0 ? 0LL : (long long)w.wait_limit);
    cudaError_t le = cudaLaunchKernelEx(&cfg, k_trsv_cl<LOWER>, N, nblk, LU, ld, v, perm, dinv, out, w.err, wait, w.rs);
    prof_end("k_trsv_cl", st);
    NL_CUDA_OK(le);
    return NL_OK;
}

nl_status trsv_solve16(int N, const __half* LU, int64_t ld, const float* v, float* z, const TrsvWork& w, int epoch,
                       cudaStream_t st, int* launches)
{
    const int C = trsv_cluster_size((int)cdiv(N, T2), w.cluster);
    if (C > 0) {
        float* y = (float*)w.y;
        nl_status s = launch_trsv_cl<true>(N, LU, ld, v, y, w, C, st);
        if (s == NL_OK) s = launch_trsv_cl<false>(N, LU, ld, y, z, w, C, st);
        if (launches) *launches += 2;
        return s;
    }
    unsigned long long* mbf = (unsigned long long*)w.y;
    unsigned long long* mbb = mbf + N;
    nl_status s = launch_trsv_mb<true>(N, LU, ld, v, nullptr, mbf, nullptr, w, (unsigned)epoch, st);
    if (s != NL_OK) return s;
    s = launch_trsv_mb<false>(N, LU, ld, nullptr, mbf, mbb, z, w, (unsigned)epoch, st);
    if (launches) *launches += 2;
    return s;
}

nl_status trsv_solve64(int N, const double* LU, int64_t ld, const double* v, double* z, const TrsvWork& w, int epoch,
                       cudaStream_t st, int* launches)
{
    return solve_impl<double, double>(N, LU, ld, v, z, w, epoch, st, launches);
}

nl_status trsv_solve32(int N, const float* LU, int64_t ld, const float* v, float* z, const TrsvWork& w, int epoch,
                       cudaStream_t st, int* launches)
{
    return solve_impl<float, float>(N, LU, ld, v, z, w, epoch, st, launches);
}

// The binary16 factors promoted to a single-precision copy (exact), for the
// GMRES-IR preconditioner that solves with single-precision factors.
__global__ void __launch_bounds__(256) k_promote16(int N, const __half* __restrict__ A, int64_t lda,
                                                   float* __restrict__ B, int64_t ldb)
{
    const int64_t i = blockIdx.y;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x)
        B[i * ldb + j] = __half2float(A[i * lda + j]);
}

nl_status launch_promote16(int N, const __half* A, int64_t lda, float* B, int64_t ldb, cudaStream_t st)
{
    if (N < 1 || N > 32768) return NL_EINVAL;
    k_promote16<<<dim3((unsigned)std::min<int64_t>(cdiv(N, 256), 8), (unsigned)N), 256, 0, st>>>(N, A, lda, B, ldb);
    NL_CUDA_OK(cudaGetLastError());
    return NL_OK;
}

// ------------------------------------------------- binary16 arithmetic --
// Both triangular solves with every product and difference rounded to
// binary16: the step of the two-precision F16 Newton method (Section 1.3),
// computed in the precision of its factorisation.  Column-oriented in one
// CTA: at step t the final entry x_t is applied to every later row (forward)
// or earlier row (backward), so row i takes its updates in increasing t in
// the forward solve and in decreasing t in the backward one.  The product of
// two binary16 numbers is exact in binary32 and is rounded once, to binary16;
// the difference and the backward quotient are formed in binary32 (IEEE
// round to nearest) and then rounded to binary16, which gives the correctly
// rounded binary16 result because 24 >= 2 * 11 + 2 (rounding twice is
// innocuous when the wider format has at least 2p + 2 bits, Figueroa 1995).
// All in single precision: binary64 here would run on the SM's few FP64
// units and dominate the sweep.
constexpr int kH16Threads = 1024;

__device__ __forceinline__ __half h16_sub_prod(__half b, __half l, __half x)
{
    const float p = __half2float(__float2half_rn(__half2float(l) * __half2float(x)));
    return __float2half_rn(__half2float(b) - p);
}

__device__ __forceinline__ __half h16_div(__half a, __half b)
{
    return __float2half_rn(__fdiv_rn(__half2float(a), __half2float(b)));
}

// Register-pipelined sweep for N <= 4096 (R <= 4 rows per thread, row
// i = tid + k * 1024): the factor is read in chunks of eight columns, one
// 16-byte load per row and chunk, issued a chunk ahead of its use, so the
// loads overlap the previous chunk's eight barrier steps.  Same operations in
// the same order as the scalar sweep.
__device__ __forceinline__ __half h16_lane(const uint4& v, int s)
{
    const unsigned w = (s >> 1) == 0 ? v.x : (s >> 1) == 1 ? v.y : (s >> 1) == 2 ? v.z : v.w;
    return __ushort_as_half((unsigned short)(w >> (16 * (s & 1))));
}

template <int R>
__device__ __forceinline__ void h16_load_chunk(const __half* __restrict__ LU, int64_t ld, int N, int c, int tid,
                                               uint4 (&v)[R])
{
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int i = tid + k * kH16Threads;
        v[k] = (i < N && c >= 0 && 8 * c < N) ? __ldg(reinterpret_cast<const uint4*>(LU + (int64_t)i * ld + 8 * c))
                                              : make_uint4(0u, 0u, 0u, 0u);
    }
}

// u_tt for t in [8c, 8c + 8) (1 beyond N), packed as one 16-byte value.
__device__ __forceinline__ uint4 h16_load_diag(const __half* __restrict__ LU, int64_t ld, int N, int c)
{
    unsigned w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int t0 = 8 * c + 2 * q, t1 = t0 + 1;
        const unsigned short lo = (c >= 0 && t0 < N) ? __half_as_ushort(LU[(int64_t)t0 * ld + t0]) : (unsigned short)0x3c00;
        const unsigned short hi = (c >= 0 && t1 < N) ? __half_as_ushort(LU[(int64_t)t1 * ld + t1]) : (unsigned short)0x3c00;
        w[q] = (unsigned)lo | ((unsigned)hi << 16);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

template <int R>
__device__ void lusolve16h_vec(int N, const __half* __restrict__ LU, int64_t ld, __half* b, __half* zout,
                               float* __restrict__ u, float scale, int tid)
{
    const int nch = (N + 7) / 8;
    uint4 cur[R], nxt[R];
    h16_load_chunk<R>(LU, ld, N, 0, tid, cur);
    for (int c = 0; c < nch; ++c) {  // L y = P b, unit diagonal
        h16_load_chunk<R>(LU, ld, N, c + 1, tid, nxt);
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const int t = 8 * c + s;
            if (t < N - 1) {
                const __half xt = b[t];
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const int i = tid + k * kH16Threads;
                    if (i > t && i < N) b[i] = h16_sub_prod(b[i], h16_lane(cur[k], s), xt);
                }
                __syncthreads();
            }
        }
#pragma unroll
        for (int k = 0; k < R; ++k) cur[k] = nxt[k];
    }
    // the chunk's diagonal entries u_tt, packed eight binary16 to 16 bytes
    uint4 dcur = h16_load_diag(LU, ld, N, nch - 1), dnxt;
    h16_load_chunk<R>(LU, ld, N, nch - 1, tid, cur);
    for (int c = nch - 1; c >= 0; --c) {  // U z = y
        h16_load_chunk<R>(LU, ld, N, c - 1, tid, nxt);
        dnxt = h16_load_diag(LU, ld, N, c - 1);
#pragma unroll
        for (int s = 7; s >= 0; --s) {
            const int t = 8 * c + s;
            if (t < N) {
                const __half xt = h16_div(b[t], h16_lane(dcur, s));
                if (tid == 0) {
                    if (zout) zout[t] = xt;
                    if (u) u[t] = scale * __half2float(xt);
                }
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const int i = tid + k * kH16Threads;
                    if (i < t) b[i] = h16_sub_prod(b[i], h16_lane(cur[k], s), xt);
                }
                __syncthreads();
            }
        }
#pragma unroll
        for (int k = 0; k < R; ++k) cur[k] = nxt[k];
        dcur = dnxt;
    }
}

__global__ void __launch_bounds__(kH16Threads) k_lusolve16h(int N, const __half* __restrict__ LU, int64_t ld,
                                                           const int* __restrict__ ipiv, const int* __restrict__ perm,
                                                           const double* __restrict__ F, const float* __restrict__ r,
                                                           const double* __restrict__ nrm, const __half* vin,
                                                           __half* zout, float* __restrict__ u)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __half* b = reinterpret_cast<__half*>(smem_raw);  // N entries
    const int tid = threadIdx.x;
    float scale = 1.0f;
    if (F) {
        const double fn = *nrm;
        for (int i = tid; i < N; i += kH16Threads) {
            const int j = perm ? perm[i] : i;
            b[i] = __double2half(-F[j] / fn);
        }
    } else if (r) {
        scale = (float)*nrm;
        for (int i = tid; i < N; i += kH16Threads) {
            const int j = perm ? perm[i] : i;
            b[i] = __float2half_rn(r[j] / scale);
        }
    } else {
        for (int i = tid; i < N; i += kH16Threads) b[i] = vin[perm ? perm[i] : i];
    }
    __syncthreads();
    if (!perm && tid == 0) {  // P b, the interchanges in factorisation order
        for (int k = 0; k < N; ++k) {
            const int p = ipiv[k];
            if (p != k && (unsigned)p < (unsigned)N) {
                const __half t = b[k];
                b[k] = b[p];
                b[p] = t;
            }
        }
    }
    __syncthreads();
    const bool vec = N <= 4 * kH16Threads && (ld % 8) == 0 && (((uintptr_t)LU) & 15) == 0;
    if (vec) {
        const int R = (N + kH16Threads - 1) / kH16Threads;
        if (R == 1) lusolve16h_vec<1>(N, LU, ld, b, zout, u, scale, tid);
        else if (R == 2) lusolve16h_vec<2>(N, LU, ld, b, zout, u, scale, tid);
        else lusolve16h_vec<4>(N, LU, ld, b, zout, u, scale, tid);
        return;
    }
    for (int t = 0; t + 1 < N; ++t) {  // L y = P b, unit diagonal
        const __half xt = b[t];
        for (int i = t + 1 + tid; i < N; i += kH16Threads) b[i] = h16_sub_prod(b[i], LU[(int64_t)i * ld + t], xt);
        __syncthreads();
    }
    for (int t = N - 1; t >= 0; --t) {  // U z = y
        const __half xt = h16_div(b[t], LU[(int64_t)t * ld + t]);
        if (tid == 0) {
            if (zout) zout[t] = xt;
            if (u) u[t] = scale * __half2float(xt);
        }
        for (int i = tid; i < t; i += kH16Threads) b[i] = h16_sub_prod(b[i], LU[(int64_t)i * ld + t], xt);
        __syncthreads();
    }
}

nl_status lusolve16h(int N, const __half* LU, int64_t ld, const int* ipiv, const int* perm, const double* F,
                     const float* r, const double* nrm, const __half* vin, __half* zout, float* u, cudaStream_t st)
{
    if (N < 1 || N > 32768 || !LU || !(ipiv || perm) || ld < N || ((F || r) ? !nrm : !vin)) {
        set_error("binary16 solve: bad argument");
        return NL_EINVAL;
    }
    static bool attr = false;
    if (!attr) {
        if (set_max_dynamic_smem((const void*)k_lusolve16h) != NL_OK) return NL_ECUDA;
        attr = true;
    }
    prof_begin("k_lusolve16h", st);
    k_lusolve16h<<<1, kH16Threads, (size_t)N * sizeof(__half), st>>>(N, LU, ld, ipiv, perm, F, r, nrm, vin, zout, u);
    prof_end("k_lusolve16h", st);
    NL_CUDA_OK(cudaGetLastError());
    return NL_OK;
}

}  // namespace nl
