// lu.cu — blocked right-looking LU with partial pivoting (Section 1.3:
// Gaussian elimination; Section 2: the half-precision factorisation of J_h).
//
// Two-level blocking.  The matrix is processed in outer panels of NB columns.
// Each outer panel is copied into a working array P (binary32 for the
// half-precision LU, binary64 for the double LU) and factored leaf by leaf
// (leaf = kLeaf columns):
//   * k_leaf: one thread-block cluster holds the leaf's rows in registers.
//     Per column, each CTA finds its best pivot candidate (warp shuffles),
//     broadcasts the candidate row to every CTA of the cluster through
//     distributed shared memory, and after one cluster barrier every CTA
//     picks the same pivot (largest |a|, first in the current row order)
//     and eliminates.  Rows stay in place; positions are tracked, and the
//     rows are written to their final positions at the end.  The epilogue
//     applies the leaf's interchanges to the other panel columns and forms
//     the leaf's U rows for the remaining panel columns.
//   * k_panel_gemm: the rest of the panel below the leaf is updated.
// After the panel: interchanges on the other columns of the matrix (k_laswp),
// U12 = L11^{-1} A12 (k_trsm_u12), and the trailing update
// A22 <- A22 - L21 U12 (SIMT here, or tcgen05 in gemm_tc.cu).
//
// Half-precision arithmetic model: binary32 arithmetic on binary16 data; the
// multipliers and the pivot rows' entries are rounded to binary16 as soon as
// they are formed, and everything not yet eliminated is rounded to binary16
// once per outer panel (when P is written back and when the trailing update
// is stored).  With the SIMT trailing update this reproduces, operation for
// operation, Gaussian elimination with that rounding schedule.
#include <atomic>
#include <cooperative_groups.h>

#include <algorithm>
#include <climits>
#include <queue>
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "tcgen05.cuh"

namespace cg = cooperative_groups;

namespace nl {

constexpr int kLeafThreads = 256;
constexpr int kMaxCluster = 16;

template <typename T, int NBL>
struct alignas(16) LeafRec {
    T abs;      // |candidate|, -1 when the CTA has no live row
    int pos;    // candidate's current position (relative to the leaf's first row)
    int pad;
    T v[NBL];   // candidate row over the leaf's columns
};

template <typename T>
__device__ __forceinline__ bool better(T a, int pa, T b, int pb)
{
    return a > b || (a == b && pa < pb);
}

template <typename T>
__device__ __forceinline__ T maybe_round(T v, bool r)
{
    return v;
}
template <>
__device__ __forceinline__ float maybe_round<float>(float v, bool r)
{
    return r ? round_h(v) : v;
}

// Register-array element at a runtime index, by static selects (keeps the
// array in registers).
template <int NBL, typename T>
__device__ __forceinline__ T pick(const T (&row)[NBL], int j)
{
    T r = row[0];
#pragma unroll
    for (int t = 1; t < NBL; ++t)
        if (t == j) r = row[t];
    return r;
}
template <int NBL, typename T>
__device__ __forceinline__ void place(T (&row)[NBL], int j, T v)
{
#pragma unroll
    for (int t = 0; t < NBL; ++t)
        if (t == j) row[t] = v;
}

// P: working panel, row r (relative to the panel's first row K), column t
// (relative to K), leading dimension ldp.  The leaf covers columns
// [k0, k0+wl) and rows [k0, M).  ipiv_out points at ipiv[K + k0].
template <typename T, int NBL, int R, bool RND>
__global__ void __launch_bounds__(kLeafThreads, 1) k_leaf(T* __restrict__ P, int ldp, int k0, int M, int w, int wl,
                                                       int* __restrict__ ipiv_out, int piv_base,
                                                       int* __restrict__ info, int C, int rows_per_cta)
{
    using Rec = LeafRec<T, NBL>;
    __shared__ Rec inbox[2][kMaxCluster];
    __shared__ Rec outbox;
    __shared__ Rec prow_save[NBL];  // pivot row of each step: L11 (below diag) and U11
    __shared__ T wabs[kLeafThreads / 32];
    __shared__ int wpos[kLeafThreads / 32];
    __shared__ int piv_s[NBL];

    const int rank = (C > 1) ? (int)cg::this_cluster().block_rank() : 0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int Ml = M - k0;
    const int lo = rank * rows_per_cta, hi = min(Ml, lo + rows_per_cta);

    T v[R][NBL];
    int pos[R];
    bool live[R];
#pragma unroll
    for (int s = 0; s < R; ++s) {
        int lr = lo + tid + s * kLeafThreads;
        live[s] = lr < hi;
        pos[s] = lr;
#pragma unroll
        for (int t = 0; t < NBL; ++t)
            v[s][t] = (live[s] && t < wl) ? P[(int64_t)(k0 + lr) * ldp + k0 + t] : T(0);
    }

    for (int j = 0; j < wl; ++j) {
        // ---- local and CTA-wide candidate: largest |a_ij|, then smallest position
        T babs = T(-1);
        int bpos = INT_MAX, bs = -1;
#pragma unroll
        for (int s = 0; s < R; ++s) {
            if (live[s]) {
                T a = pick<NBL>(v[s], j);
                a = a < T(0) ? -a : a;
                if (!(a == a)) a = T(-0.5);  // NaN never wins over a number
                if (better(a, pos[s], babs, bpos)) {
                    babs = a;
                    bpos = pos[s];
                    bs = s;
                }
            }
        }
        T wa = babs;
        int wp = bpos;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            T oa = __shfl_xor_sync(0xffffffffu, wa, o);
            int op = __shfl_xor_sync(0xffffffffu, wp, o);
            if (better(oa, op, wa, wp)) {
                wa = oa;
                wp = op;
            }
        }
        if (lane == 0) {
            wabs[warp] = wa;
            wpos[warp] = wp;
        }
        __syncthreads();
        T ca = T(-1);
        int cp = INT_MAX;
        for (int q = 0; q < kLeafThreads / 32; ++q)
            if (better(wabs[q], wpos[q], ca, cp)) {
                ca = wabs[q];
                cp = wpos[q];
            }
        if (bs >= 0 && bpos == cp) {
            outbox.abs = ca;
            outbox.pos = cp;
#pragma unroll
            for (int s = 0; s < R; ++s)
                if (s == bs) {
#pragma unroll
                    for (int t = 0; t < NBL; ++t) outbox.v[t] = v[s][t];
                }
        }
        if (cp == INT_MAX && tid == 0) {
            outbox.abs = T(-1);
            outbox.pos = INT_MAX;
        }
        __syncthreads();

        // ---- exchange candidates across the cluster
        const Rec* recs;
        int nrec;
        if (C > 1) {
            cg::cluster_group cl = cg::this_cluster();
            constexpr int kWords = sizeof(Rec) / 16;
            for (int q = tid; q < C * kWords; q += kLeafThreads) {
                int peer = q / kWords, wd = q % kWords;
                float4* dst = reinterpret_cast<float4*>(cl.map_shared_rank(&inbox[j & 1][rank], peer));
                dst[wd] = reinterpret_cast<const float4*>(&outbox)[wd];
            }
            cl.sync();
            recs = inbox[j & 1];
            nrec = C;
        } else {
            recs = &outbox;
            nrec = 1;
        }
        T ga = T(-1);
        int gp = INT_MAX, gsrc = 0;
        for (int q = 0; q < nrec; ++q)
            if (better(recs[q].abs, recs[q].pos, ga, gp)) {
                ga = recs[q].abs;
                gp = recs[q].pos;
                gsrc = q;
            }
        const Rec& pr = recs[gsrc];
        T u[NBL];
#pragma unroll
        for (int t = 0; t < NBL; ++t) u[t] = (t >= j) ? maybe_round(pr.v[t], RND) : T(0);
        if (tid == 0) {
            piv_s[j] = gp;
            if (rank == 0) ipiv_out[j] = piv_base + gp;
            // keep the pivot row: entries left of j are its multipliers
#pragma unroll
            for (int t = 0; t < NBL; ++t) prow_save[j].v[t] = (t >= j) ? u[t] : pr.v[t];
        }

        // ---- interchange bookkeeping: the pivot row moves to position j,
        //      the row at position j moves to the pivot's old position
#pragma unroll
        for (int s = 0; s < R; ++s) {
            if (live[s]) {
                if (pos[s] == gp) {
                    live[s] = false;
                    pos[s] = j;
#pragma unroll
                    for (int t = 0; t < NBL; ++t)
                        if (t >= j) v[s][t] = u[t];
                } else if (pos[s] == j) {
                    pos[s] = gp;
                }
            }
        }

        // ---- elimination of column j in the live rows
        const T ukk = pick<NBL>(u, j);
        if (ukk != T(0)) {
#pragma unroll
            for (int s = 0; s < R; ++s) {
                if (live[s]) {
                    T l = maybe_round(pick<NBL>(v[s], j) / ukk, RND);
                    place<NBL>(v[s], j, l);
#pragma unroll
                    for (int t = 0; t < NBL; ++t)
                        if (t > j) v[s][t] = fma(-l, u[t], v[s][t]);
                }
            }
        } else if (tid == 0 && rank == 0) {
            atomicCAS(info, 0, piv_base + j + 1);
        }
    }

    // ---- rows to their final positions (leaf columns)
#pragma unroll
    for (int s = 0; s < R; ++s) {
        int lr = lo + tid + s * kLeafThreads;
        if (lr < hi) {
#pragma unroll
            for (int t = 0; t < NBL; ++t)
                if (t < wl) P[(int64_t)(k0 + pos[s]) * ldp + k0 + t] = v[s][t];
        }
    }
    if (rank != 0) return;
    __syncthreads();

    // ---- epilogue (one CTA): interchanges on the other panel columns, then
    //      the leaf's U rows for the panel columns right of the leaf
    const int nother = w - wl;
    for (int q = tid; q < nother; q += kLeafThreads) {
        int col = (q < k0) ? q : q + wl;
        for (int jj = 0; jj < wl; ++jj) {
            int p = piv_s[jj];
            if (p != jj) {
                T* a = P + (int64_t)(k0 + jj) * ldp + col;
                T* b = P + (int64_t)(k0 + p) * ldp + col;
                T tmp = *a;
                *a = *b;
                *b = tmp;
            }
        }
        if (col >= k0 + wl) {
            T uu[NBL];
#pragma unroll
            for (int kk = 0; kk < NBL; ++kk) {
                if (kk < wl) {
                    T a = P[(int64_t)(k0 + kk) * ldp + col];
#pragma unroll
                    for (int t = 0; t < NBL; ++t)
                        if (t < kk) a = fma(-prow_save[kk].v[t], uu[t], a);
                    a = maybe_round(a, RND);
                    uu[kk] = a;
                    P[(int64_t)(k0 + kk) * ldp + col] = a;
                } else {
                    uu[kk] = T(0);
                }
            }
        }
    }
}

// Rest of the panel below a leaf: P[i][c] -= sum_t P[i][k0+t] P[k0+t][c],
// rows i in [k0+wl, M), columns c in [k0+wl, w), t in [0, wl) in order,
// kept in the working precision (no rounding).
template <typename T, int NBL>
__global__ void __launch_bounds__(256) k_panel_gemm(T* __restrict__ P, int ldp, int k0, int wl, int M, int w)
{
    __shared__ T Us[NBL][64];
    const int c0 = k0 + wl;
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
    const int rbase = c0 + blockIdx.x * 64;
    for (int cc = 0; cc < w - c0; cc += 64) {
        const int c = c0 + cc + tx;
        __syncthreads();
        for (int q = threadIdx.x; q < NBL * 64; q += 256) {
            int t = q / 64, x = q % 64;
            Us[t][x] = (t < wl && c0 + cc + x < w) ? P[(int64_t)(k0 + t) * ldp + c0 + cc + x] : T(0);
        }
        __syncthreads();
        if (c < w) {
            for (int rr = ty; rr < 64; rr += 4) {
                int i = rbase + rr;
                if (i >= M) break;
                const T* Li = P + (int64_t)i * ldp + k0;
                T acc = P[(int64_t)i * ldp + c];
#pragma unroll
                for (int t = 0; t < NBL; ++t)
                    if (t < wl) acc = fma(-Li[t], Us[t][tx], acc);
                P[(int64_t)i * ldp + c] = acc;
            }
        }
    }
}

template <typename T, typename S>
__global__ void k_panel_load(const S* __restrict__ A, int64_t lda, int K, int M, int w, T* __restrict__ P, int ldp)
{
    const int i = blockIdx.x;
    for (int t = threadIdx.x; t < w; t += blockDim.x) P[(int64_t)i * ldp + t] = (T)ld_elem(A + (int64_t)(K + i) * lda + K + t);
}

template <typename T, typename S>
__global__ void k_panel_store(S* __restrict__ A, int64_t lda, int K, int M, int w, const T* __restrict__ P, int ldp)
{
    const int i = blockIdx.x;
    for (int t = threadIdx.x; t < w; t += blockDim.x) st_elem(A + (int64_t)(K + i) * lda + K + t, P[(int64_t)i * ldp + t]);
}

// Row interchanges of panel [K, K+w) on all other columns, in order.
template <typename S>
__global__ void __launch_bounds__(256) k_laswp(S* __restrict__ A, int64_t lda, int K, int w, int N,
                                               const int* __restrict__ ipiv)
{
    __shared__ int ps[256];
    for (int q = threadIdx.x; q < w; q += blockDim.x) ps[q] = ipiv[K + q];
    __syncthreads();
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= N - w) return;
    const int col = (q < K) ? q : q + w;
    for (int jj = 0; jj < w; ++jj) {
        int p = ps[jj];
        if (p != K + jj) {
            S* a = A + (int64_t)(K + jj) * lda + col;
            S* b = A + (int64_t)p * lda + col;
            S t = *a;
            *a = *b;
            *b = t;
        }
    }
}

// U12 = L11^{-1} A12 for rows [K, K+w), columns [K+w, N); each thread forms
// one column by forward substitution, rounding each entry when formed (half
// LU).  Rows are taken eight at a time so that the eight running sums are
// independent (instruction-level parallelism); each entry still accumulates
// its terms t = 0, 1, ..., k-1 in order.  Optionally also writes U12^T
// (binary16, ldut) for the tensor-core update.  flag: skip when set.
constexpr int kTrsmThreads = 64;

template <typename T, typename S, bool RND>
__global__ void __launch_bounds__(kTrsmThreads) k_trsm_u12(S* __restrict__ A, int64_t lda, int K, int w, int N,
                                                          __half* __restrict__ Ut, int ldut,
                                                          const int* __restrict__ flag)
{
    if (flag && *(volatile const int*)flag) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* L = reinterpret_cast<T*>(smem_raw);  // w x w, strictly lower part
    T* us = L + w * w;                       // w x kTrsmThreads (column per thread)
    for (int q = threadIdx.x; q < w * w; q += blockDim.x) {
        int r = q / w, t = q % w;
        L[q] = (t < r) ? (T)ld_elem(A + (int64_t)(K + r) * lda + K + t) : T(0);
    }
    __syncthreads();
    const int c0 = K + w + blockIdx.x * kTrsmThreads;
    const int c = c0 + threadIdx.x;
    const int tid = threadIdx.x;
    if (c < N) {
        for (int k0 = 0; k0 < w; k0 += 8) {
            T acc[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q] = (k0 + q < w) ? (T)ld_elem(A + (int64_t)(K + k0 + q) * lda + c) : T(0);
            for (int t = 0; t < k0; ++t) {
                const T ut = us[t * kTrsmThreads + tid];
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[q] = fma(-L[(k0 + q) * w + t], ut, acc[q]);
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int k = k0 + q;
                if (k < w) {
                    T a = acc[q];
                    for (int t = k0; t < k; ++t) a = fma(-L[k * w + t], us[t * kTrsmThreads + tid], a);
                    a = maybe_round(a, RND);
                    us[k * kTrsmThreads + tid] = a;
                    st_elem(A + (int64_t)(K + k) * lda + c, a);
                }
            }
        }
    }
    if (Ut) {
        __syncthreads();
        const int ncol = min(kTrsmThreads, N - c0);
        for (int q = threadIdx.x; q < ncol * w; q += blockDim.x) {
            int col = q / w, kk = q % w;
            Ut[(int64_t)(c0 - K - w + col) * ldut + kk] = __float2half_rn((float)us[kk * kTrsmThreads + col]);
        }
    }
}

// ------------------------------------------------ no-interchange fast path --
// Partial pivoting picks the diagonal row at step j exactly when no row
// below holds a larger |a_ij| (ties go to the diagonal, which comes first).
// The fast path factors each panel without interchanges and checks that
// condition on every pre-division value; the elimination arithmetic is the
// same, so when no check fails the factors and pivots (ipiv[k] = k) are
// exactly those of partial pivoting.  Any failure (or a zero / NaN pivot)
// sets *flag; the remaining fast-path kernels then return at once and the
// caller refactors with the interchanging path.

// ------------------------------------------------ 32-wide chunk routines --
// All routines below apply to each entry the elimination's updates
// a <- a - l_t u_t in increasing t (one rounding each: the product of two
// binary16 numbers is exact in binary32), round multipliers and U entries to
// binary16 when they are formed, and check each pre-division value against
// its pivot (|a_it| <= |u_tt|: partial pivoting keeps the diagonal).

__device__ __forceinline__ float absT(float x) { return fabsf(x); }
__device__ __forceinline__ double absT(double x) { return fabs(x); }

// Diagonal block [K, K+w)^2 (w <= 128) in one CTA, held in shared memory,
// in 32-column chunks c (padding beyond w is identity):
//  (a) one warp factors the 32 x 32 diagonal sub-block, lane r = row r: at
//      step t row t is final, its U entries are rounded, and the rows below
//      form their multipliers and update;
//  (b) groups of eight lanes solve the rows below the sub-block against its
//      U, and (c) the columns right of it against its L (as k_offdiag does);
//  (d) all threads apply the rank-32 update to the rest of the block.
constexpr int kDiagThreads = 512;
constexpr int kOffG = 8;  // lanes per row / column group

// Block [K, K+w)^2 of A into shared memory W (ld ldw), identity-padded to
// wp; 16-byte vector loads when the row segments allow them.
template <typename T, typename S, int NT>
__device__ __forceinline__ void load_block(const S* __restrict__ A, int64_t lda, int K, int w, int wp, T* W, int ldw,
                                           int tid)
{
    constexpr int V = 16 / sizeof(S);  // elements per 16-byte vector
    const bool vec = (w % V == 0) && ((((uintptr_t)(A + (int64_t)K * lda + K)) & 15) == 0) && ((lda * sizeof(S)) % 16 == 0);
    if (vec) {
        const int vpr = w / V;
#pragma unroll 4
        for (int q = tid; q < w * vpr; q += NT) {
            const int i = q / vpr, tv = q - i * vpr;
            uint4 raw = *reinterpret_cast<const uint4*>(A + (int64_t)(K + i) * lda + K + tv * V);
            const S* e = reinterpret_cast<const S*>(&raw);
#pragma unroll
            for (int k = 0; k < V; ++k) W[i * ldw + tv * V + k] = (T)ld_elem(e + k);
        }
    } else {
#pragma unroll 4
        for (int q = tid; q < w * w; q += NT) {
            const int i = q / w, t = q - i * w;
            W[i * ldw + t] = (T)ld_elem(A + (int64_t)(K + i) * lda + K + t);
        }
    }
    for (int q = tid; q < wp * wp; q += NT) {
        const int i = q / wp, t = q - i * wp;
        if (i >= w || t >= w) W[i * ldw + t] = (i == t) ? T(1) : T(0);
    }
}

template <typename T, typename S, int NT>
__device__ __forceinline__ void store_block(S* __restrict__ A, int64_t lda, int K, int w, const T* W, int ldw, int tid)
{
    constexpr int V = 16 / sizeof(S);
    const bool vec = (w % V == 0) && ((((uintptr_t)(A + (int64_t)K * lda + K)) & 15) == 0) && ((lda * sizeof(S)) % 16 == 0);
    if (vec) {
        const int vpr = w / V;
#pragma unroll 4
        for (int q = tid; q < w * vpr; q += NT) {
            const int i = q / vpr, tv = q - i * vpr;
            uint4 raw;
            S* e = reinterpret_cast<S*>(&raw);
#pragma unroll
            for (int k = 0; k < V; ++k) st_elem(e + k, W[i * ldw + tv * V + k]);
            *reinterpret_cast<uint4*>(A + (int64_t)(K + i) * lda + K + tv * V) = raw;
        }
    } else {
        for (int q = tid; q < w * w; q += NT) {
            const int i = q / w, t = q - i * w;
            st_elem(A + (int64_t)(K + i) * lda + K + t, W[i * ldw + t]);
        }
    }
}

template <typename T, bool RND>
__device__ __forceinline__ void group_row_solve(T* W, int ldw, int c0, int r, int g, unsigned gmask, bool& bad)
{
    // row r, chunk columns c0 + 4g .. c0 + 4g + 3, against U = W[c0.., c0..]
    T acc[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] = W[r * ldw + c0 + 4 * g + k];
#pragma unroll
    for (int tt = 0; tt < 32; ++tt) {
        T l = T(0);
        if (g == tt / 4) {
            const T utt = W[(c0 + tt) * ldw + c0 + tt];
            const T x = acc[tt % 4];
            if (!(absT(x) <= absT(utt)) || !(utt != T(0))) bad = true;
            l = maybe_round(x / utt, RND);
            acc[tt % 4] = l;
        }
        l = __shfl_sync(gmask, l, tt / 4, kOffG);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (4 * g + k > tt) acc[k] = fma(-l, W[(c0 + tt) * ldw + c0 + 4 * g + k], acc[k]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) W[r * ldw + c0 + 4 * g + k] = acc[k];
}

template <typename T, bool RND>
__device__ __forceinline__ void group_col_solve(T* W, int ldw, int c0, int col, int g, unsigned gmask)
{
    // column col, chunk rows c0 + 4g .. c0 + 4g + 3, against L = W[c0.., c0..]
    T acc[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] = W[(c0 + 4 * g + k) * ldw + col];
#pragma unroll
    for (int tt = 0; tt < 32; ++tt) {
        T u = T(0);
        if (g == tt / 4) {
            u = maybe_round(acc[tt % 4], RND);
            acc[tt % 4] = u;
        }
        u = __shfl_sync(gmask, u, tt / 4, kOffG);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (4 * g + k > tt) acc[k] = fma(-W[(c0 + 4 * g + k) * ldw + c0 + tt], u, acc[k]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) W[(c0 + 4 * g + k) * ldw + col] = acc[k];
}

template <typename T, typename S, bool RND>
__device__ __forceinline__ void diag_lu_body(S* __restrict__ A, int64_t lda, int K, int w,
                                                             int* __restrict__ ipiv, int* __restrict__ flag,
                                                             void* __restrict__ stage)
{
    if (*(volatile int*)flag) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* W = reinterpret_cast<T*>(smem_raw);
    const int wp = (w + 31) & ~31, ldw = wp + 1;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int grp = tid / kOffG, g = tid % kOffG;
    const unsigned gmask = 0xffu << ((tid & 31) & ~(kOffG - 1));
    load_block<T, S, kDiagThreads>(A, lda, K, w, wp, W, ldw, tid);
    __syncthreads();
    bool bad = false;
    const int nc = wp / 32;
    for (int c = 0; c < nc; ++c) {
        const int c0 = 32 * c;
        if (warp == 0) {
            // lane r holds row c0 + r of the sub-block; after step t the row
            // array is shifted by one so that a[0] is always column c0 + t
            T* Wr = W + (c0 + lane) * ldw + c0;
            T a[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) a[j] = Wr[j];
            for (int t = 0; t < 32; ++t) {
                const T utt = __shfl_sync(0xffffffffu, maybe_round(a[0], RND), t);
                // rows below form their multiplier; finished rows use l = 0
                T l = T(0);
                if (lane > t) {
                    if (!(absT(a[0]) <= absT(utt)) || !(utt != T(0))) bad = true;
                    l = maybe_round(a[0] / utt, RND);
                }
                a[0] = (lane == t) ? utt : ((lane > t) ? l : a[0]);
                if (lane >= t) Wr[t] = a[0];
#pragma unroll
                for (int j = 1; j < 32; ++j) {
                    const T uj = __shfl_sync(0xffffffffu, maybe_round(a[j], RND), t);
                    a[j] = (lane == t) ? uj : fma(-l, uj, a[j]);
                }
                if (lane == t) {
#pragma unroll
                    for (int j = 1; j < 32; ++j)
                        if (t + j < 32) Wr[t + j] = a[j];  // U entries of row t
                }
#pragma unroll
                for (int j = 0; j < 31; ++j) a[j] = a[j + 1];
                a[31] = T(0);
            }
        }
        __syncthreads();
        const int rest = wp - c0 - 32;
        // (b) rows below and (c) columns right of the sub-block: one group each
        for (int q = grp; q < 2 * rest; q += kDiagThreads / kOffG) {
            if (q < rest) group_row_solve<T, RND>(W, ldw, c0, c0 + 32 + q, g, gmask, bad);
            else group_col_solve<T, RND>(W, ldw, c0, c0 + 32 + (q - rest), g, gmask);
        }
        __syncthreads();
        if (rest > 0) {
            // (d) rows/cols [c0+32, wp): 2 x 2 entries per thread, t in order
            const int nb2 = rest / 2;
            for (int e = tid; e < nb2 * nb2; e += kDiagThreads) {
                const int i = c0 + 32 + 2 * (e / nb2), j = c0 + 32 + 2 * (e % nb2);
                T a00 = W[i * ldw + j], a01 = W[i * ldw + j + 1];
                T a10 = W[(i + 1) * ldw + j], a11 = W[(i + 1) * ldw + j + 1];
#pragma unroll 8
                for (int t = c0; t < c0 + 32; ++t) {
                    const T l0 = W[i * ldw + t], l1 = W[(i + 1) * ldw + t];
                    const T u0 = W[t * ldw + j], u1 = W[t * ldw + j + 1];
                    a00 = fma(-l0, u0, a00);
                    a01 = fma(-l0, u1, a01);
                    a10 = fma(-l1, u0, a10);
                    a11 = fma(-l1, u1, a11);
                }
                W[i * ldw + j] = a00;
                W[i * ldw + j + 1] = a01;
                W[(i + 1) * ldw + j] = a10;
                W[(i + 1) * ldw + j + 1] = a11;
            }
            __syncthreads();
        }
    }
    if (__syncthreads_or(bad)) {
        if (tid == 0) atomicOr(flag, 1);
        return;
    }
    store_block<T, S, kDiagThreads>(A, lda, K, w, W, ldw, tid);
    // staged copies for k_offdiag: U11 (row role) and L11^T (column role),
    // wp x wp each, identity / zero padded, in its shared-memory layout
    using H = typename std::conditional<std::is_same<S, __half>::value, __half, T>::type;
    H* SU = reinterpret_cast<H*>(stage);
    H* SL = SU + wp * wp;
    for (int q = tid; q < wp * wp; q += kDiagThreads) {
        const int r = q / wp, t = q - r * wp;
        const T wv = W[r * ldw + t], wt = W[t * ldw + r];
        SU[q] = (H)((r < w && t < w) ? ((t >= r) ? wv : T(0)) : ((r == t) ? T(1) : T(0)));
        SL[q] = (H)((r < w && t < w && t > r) ? wt : T(0));
    }
    if (tid < w) ipiv[K + tid] = K + tid;
}

template <typename T, typename S, bool RND>
__global__ void __launch_bounds__(kDiagThreads, 1) k_diag_lu(S* __restrict__ A, int64_t lda, int K, int w,
                                                             int* __restrict__ ipiv, int* __restrict__ flag,
                                                             void* __restrict__ stage)
{
    diag_lu_body<T, S, RND>(A, lda, K, w, ipiv, flag, stage);
}

// Off-diagonal blocks of a panel of width w, one launch, eight lanes per row
// (L21 = A21 U11^{-1}) or per column (U12 = L11^{-1} A12), four per warp.
// Left-looking in 32-wide chunks: lane g of a group owns entries 4g..4g+3 of
// the chunk.  The chunk is first updated with the earlier chunks' multipliers
// (row role) or U entries (column role), which the group keeps in shared
// memory as binary16 (exact), then solved against the chunk's diagonal
// 32 x 32 block: at step t the owning lane forms the multiplier (or rounds
// the U entry) and broadcasts it to its group.  U11 (row role) and L11^T
// (column role) are staged in shared memory as binary16.
constexpr int kOffThreads = 128;  // 16 groups of 8 lanes

template <typename T, typename S, bool RND>
__device__ __forceinline__ void offdiag_body(S* __restrict__ A, int64_t lda, int K, int w, int N,
                                                         int nrow_blocks, __half* __restrict__ Ut, int ldut,
                                                         int* __restrict__ flag, const void* __restrict__ stage, int bid)
{
    if (flag && *(volatile int*)flag) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using H = typename std::conditional<std::is_same<S, __half>::value, __half, T>::type;
    constexpr int NG = kOffThreads / kOffG;  // groups (rows or columns) per CTA
    const int wp = (w + 31) & ~31;
    H* D = reinterpret_cast<H*>(smem_raw);  // wp x wp: U11 (row role) or L11^T (column role), identity-padded
    H* X = D + wp * wp;                     // wp x NG: earlier multipliers / U entries of each group
    const int tid = threadIdx.x, grp = tid / kOffG, g = tid % kOffG;
    const unsigned gmask = 0xffu << ((tid & 31) & ~(kOffG - 1));
    const bool row_role = (int)bid < nrow_blocks;
    {
        // U11 or L11^T, staged by k_diag_lu in exactly this layout
        const uint4* src = reinterpret_cast<const uint4*>(reinterpret_cast<const H*>(stage) + (row_role ? 0 : wp * wp));
        uint4* dst = reinterpret_cast<uint4*>(D);
        const int nv = wp * wp * (int)sizeof(H) / 16;
#pragma unroll 4
        for (int q = tid; q < nv; q += kOffThreads) dst[q] = src[q];
    }
    __syncthreads();
    bool bad = false;
    const int nc = wp / 32;
    if (row_role) {
        const int i = K + w + bid * NG + grp;
        const bool live = i < N;
        S* Ai = A + (int64_t)min(i, N - 1) * lda + K;
        for (int c = 0; c < nc; ++c) {
            const int c0 = 32 * c, jb = c0 + 4 * g;
            T acc[4];
            if (live && jb + 4 <= w) {
                S e[4];
                if constexpr (sizeof(S) == 2) *reinterpret_cast<uint2*>(e) = *reinterpret_cast<const uint2*>(Ai + jb);
                else {
                    reinterpret_cast<uint4*>(e)[0] = reinterpret_cast<const uint4*>(Ai + jb)[0];
                    reinterpret_cast<uint4*>(e)[1] = reinterpret_cast<const uint4*>(Ai + jb)[1];
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[k] = (T)ld_elem(e + k);
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[k] = (live && jb + k < w) ? (T)ld_elem(Ai + jb + k) : T(0);
            }
            for (int t = 0; t < c0; ++t) {
                const T l = (T)X[t * NG + grp];
                const H* Dt = D + t * wp + jb;
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[k] = fma(-l, (T)Dt[k], acc[k]);
            }
#pragma unroll
            for (int tt = 0; tt < 32; ++tt) {
                const int t = c0 + tt;
                T l = T(0);
                if (g == tt / 4) {
                    const T utt = (T)D[t * wp + t];
                    const T x = acc[tt % 4];
                    if (live && t < w && (!(absT(x) <= absT(utt)) || !(utt != T(0)))) bad = true;
                    l = maybe_round(x / utt, RND);
                    acc[tt % 4] = l;
                    X[t * NG + grp] = (H)l;
                }
                l = __shfl_sync(gmask, l, tt / 4, kOffG);
                const H* Dt = D + t * wp + jb;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (4 * g + k > tt) acc[k] = fma(-l, (T)Dt[k], acc[k]);
            }
            if (live) {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (jb + k < w) st_elem(Ai + jb + k, acc[k]);
            }
        }
        if (__syncthreads_or(bad) && tid == 0 && flag) atomicOr(flag, 1);
    } else {
        const int col = K + w + (bid - nrow_blocks) * NG + grp;
        const bool live = col < N;
        const int cc = min(col, N - 1);
        for (int c = 0; c < nc; ++c) {
            const int c0 = 32 * c, kb = c0 + 4 * g;
            T acc[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[k] = (live && kb + k < w) ? (T)ld_elem(A + (int64_t)(K + kb + k) * lda + cc) : T(0);
            for (int t = 0; t < c0; ++t) {
                const T u = (T)X[t * NG + grp];
                const H* Dt = D + t * wp + kb;  // L[kb + k][t]
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[k] = fma(-(T)Dt[k], u, acc[k]);
            }
#pragma unroll
            for (int tt = 0; tt < 32; ++tt) {
                const int t = c0 + tt;
                T u = T(0);
                if (g == tt / 4) {
                    u = maybe_round(acc[tt % 4], RND);
                    acc[tt % 4] = u;
                    X[t * NG + grp] = (H)u;
                }
                u = __shfl_sync(gmask, u, tt / 4, kOffG);
                const H* Dt = D + t * wp + kb;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (4 * g + k > tt) acc[k] = fma(-(T)Dt[k], u, acc[k]);
            }
            if (live) {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (kb + k < w) {
                        st_elem(A + (int64_t)(K + kb + k) * lda + col, acc[k]);
                        if (Ut) Ut[(int64_t)(col - K - w) * ldut + kb + k] = __float2half_rn((float)acc[k]);
                    }
            }
        }
    }
}

template <typename T, typename S, bool RND>
__global__ void __launch_bounds__(kOffThreads) k_offdiag(S* __restrict__ A, int64_t lda, int K, int w, int N,
                                                         int nrow_blocks, __half* __restrict__ Ut, int ldut,
                                                         int* __restrict__ flag, const void* __restrict__ stage)
{
    offdiag_body<T, S, RND>(A, lda, K, w, N, nrow_blocks, Ut, ldut, flag, stage, (int)blockIdx.x);
}

// ------------------------------------------ fast path, binary16 factors --
// The stage buffer holds, for the off-diagonal solves of one panel: U11 and
// L11^T (wp x wp binary32 each, the exact binary16 values, identity / zero
// padded) and the unrounded pivots a_tt (kStagePivOff floats in).
constexpr int kStagePivOff = 2 * 128 * 128;

// k_diag_lu16: the diagonal block [K, K+w)^2 (w <= 128), one CTA of 512
// threads, as a column pipeline.  Warp v owns columns 8v..8v+7 and lane l rows
// 4l..4l+3, so every thread keeps a 4 x 8 tile in registers.  Warp v first
// applies, in order k = 0, 1, ..., 8v-1, the updates of the earlier warps'
// columns as each column's multipliers appear in shared memory (a ready flag
// per column), then factors its own eight columns: for column t the lanes
// check |a_it| <= |a_tt| for their rows below t (partial pivoting keeps the
// diagonal; ties go to the diagonal, which comes first), form
// l_it = fl16(a_it / fl16(a_tt)), publish them, and update the warp's later
// columns.  Row k's entries of a warp's columns are rounded to binary16 (U)
// by that warp when it applies update k.  Every entry takes its updates in
// increasing k, one binary32 fused multiply-add each, exactly as in
// right-looking elimination; only the warps' schedule is pipelined, so the
// critical path is one division and one hand-off per column instead of a
// block-wide barrier per step.  Finished entries stay in the registers (U on
// and above the diagonal, L below).  Every wait is bounded: a wait that gives
// up marks the fast path failed, so the host refactors with interchanges.
// (The hand-offs use CTA-scope release/acquire on the flags; a fence per
// column and a clock-based wait cost 1.7x in time.)
constexpr int kD16Threads = 512;
constexpr size_t kDiag16Smem = 128 * 128 * sizeof(float);
constexpr int kDiagSpinLimit = 1 << 22;  // polls of a ready flag before a wait gives up

// Column hand-off inside the CTA: the producer's lane 0 publishes a column
// with a CTA-scope release store of its ready flag (shared memory); a
// consumer's lane 0 polls it with CTA-scope acquire loads, at most
// kDiagSpinLimit times.  (This exact loop shape matters: an equivalent
// for-loop with the bound test first compiled to a 2.6x slower kernel.)
__device__ __forceinline__ bool diag_wait(const int* f, int* failp)
{
    int it = 0;
    while (true) {
        int v;
        asm volatile("ld.acquire.cta.shared::cta.b32 %0, [%1];" : "=r"(v) : "r"((unsigned)__cvta_generic_to_shared(f)) : "memory");
        if (v) return true;
        if (*(volatile const int*)failp) return false;
        if (++it > kDiagSpinLimit) { *(volatile int*)failp = 1; return false; }
    }
}

// Eight consecutive entries (16-byte aligned) as binary32, and back: binary16
// storage (the factorised matrix) rounds on store; binary32 storage (the
// single-precision shadow of an outer block, two-level LU) keeps the value.
__device__ __forceinline__ void load8(const __half* p, float* v)
{
    const uint4 raw = *reinterpret_cast<const uint4*>(p);
    const __half* e = reinterpret_cast<const __half*>(&raw);
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = __half2float(e[c]);
}
__device__ __forceinline__ void load8(const float* p, float* v)
{
    const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
__device__ __forceinline__ void store8(__half* p, const float* v)
{
    __align__(16) __half h[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) h[c] = __float2half_rn(v[c]);
    *reinterpret_cast<uint4*>(p) = *reinterpret_cast<const uint4*>(h);
}
__device__ __forceinline__ void store8(float* p, const float* v)
{
    reinterpret_cast<float4*>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float4*>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
}

// PUB: also publish each finished column t to pub[t * 128 + i] as the 64-bit
// word {epoch, value} (U above the diagonal, the unrounded pivot on it, the
// multipliers below), for the streaming off-diagonal solves of k_panel16.
template <bool PUB = false, typename S = __half>
__device__ __forceinline__ void diag_lu16_body(S* __restrict__ A, int64_t lda, int K, int w,
                                               int* __restrict__ ipiv, int* __restrict__ flag,
                                               float* __restrict__ stage,
                                               unsigned long long* __restrict__ pub = nullptr, unsigned epoch = 0)
{
    if (*(volatile int*)flag) return;
    extern __shared__ __align__(16) float lsh[];  // lsh[t * 128 + i] = l_it (0 for i <= t)
    __shared__ int rdy[128];
    __shared__ int fail;
    __shared__ float pvs[128];  // unrounded pivots, copied to the stage at the end
    const int tid = threadIdx.x, lane = tid & 31, v = tid >> 5;
    const int r0 = 4 * lane, C0 = 8 * v;
    const int wp = (w + 31) & ~31;
    const bool vec = (w % 8 == 0) && ((((uintptr_t)(A + (int64_t)K * lda + K)) & 15) == 0) && (lda % 8 == 0);
    if (tid < 128) rdy[tid] = 0;
    if (tid == 0) fail = 0;
    float a[4][8];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int i = r0 + r;
        const S* src = A + (int64_t)(K + min(i, w - 1)) * lda + K + C0;
        if (vec && i < w && C0 + 8 <= w) {
            load8(src, a[r]);
        } else {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int j = C0 + c;
                a[r][c] = (i < w && j < w) ? ld_elem(src + c) : ((i == j) ? 1.0f : 0.0f);
            }
        }
    }
    __syncthreads();
    float* PV = stage + kStagePivOff;
    bool bad = false, alive = true;
    if (C0 < w) {
        // the earlier warps' columns, in order
        for (int k0 = 0; k0 < C0 && alive; k0 += 4) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const int k = k0 + kk;  // row k is register row kk of lane k / 4
                int ok = 1;
                if (lane == 0) ok = diag_wait(&rdy[k], &fail);
                __syncwarp();
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    alive = false;
                    break;
                }
                const float4 l4 = *reinterpret_cast<const float4*>(&lsh[k * 128 + r0]);
                const float lk[4] = {l4.x, l4.y, l4.z, l4.w};
                float u[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) u[c] = round_h(__shfl_sync(0xffffffffu, a[kk][c], k >> 2));
                if (lane == (k >> 2)) {
#pragma unroll
                    for (int c = 0; c < 8; ++c) a[kk][c] = u[c];
                }
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    if (r0 + r > k) {
#pragma unroll
                        for (int c = 0; c < 8; ++c) a[r][c] = fmaf(-lk[r], u[c], a[r][c]);
                    }
            }
        }
        // this warp's own columns
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            const int t = C0 + kk;
            if (alive && t < w) {
                const int src = t >> 2;  // row t is register row kk & 3 of lane t / 4
                const float p = __shfl_sync(0xffffffffu, a[kk & 3][kk], src);
                const float ut = round_h(p);
                const float rut = __frcp_rn(ut);
                float lv[4];
                bool unsure = false;
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    bool u = false;
                    lv[r] = div_round_h_fast(a[r][kk], rut, &u);
                    unsure |= u && (r0 + r > t);
                }
                if (__any_sync(0xffffffffu, unsure)) {  // rare: decide the boundary cases exactly
#pragma unroll
                    for (int r = 0; r < 4; ++r) lv[r] = div_round_h(a[r][kk], ut, rut);
                }
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    if (r0 + r > t) {
                        if (!(fabsf(a[r][kk]) <= fabsf(p))) bad = true;
                        a[r][kk] = lv[r];
                    } else {
                        lv[r] = 0.0f;
                    }
                }
                if (lane == src) {
                    a[kk & 3][kk] = ut;
                    pvs[t] = p;
                    if (!(ut != 0.0f)) bad = true;  // zero pivot: info is the interchanging path's
                }
                *reinterpret_cast<float4*>(&lsh[t * 128 + r0]) = make_float4(lv[0], lv[1], lv[2], lv[3]);
                __syncwarp();
                if (lane == 0) asm volatile("st.release.cta.shared::cta.b32 [%0], %1;" :: "r"((unsigned)__cvta_generic_to_shared(&rdy[t])), "r"(1) : "memory");
                if constexpr (PUB) {
                    // column t is final: U entries (rounded) above the diagonal, p on it, l below
                    unsigned long long wv[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int i = r0 + r;
                        const float v = (i < t) ? a[r][kk] : ((i == t) ? p : lv[r]);
                        wv[r] = ((unsigned long long)epoch << 32) | __float_as_uint(v);
                    }
                    unsigned long long* dst = pub + t * 128 + r0;
                    asm volatile("st.volatile.global.v2.u64 [%0], {%1, %2};" ::"l"(dst), "l"(wv[0]), "l"(wv[1]) : "memory");
                    asm volatile("st.volatile.global.v2.u64 [%0], {%1, %2};" ::"l"(dst + 2), "l"(wv[2]), "l"(wv[3]) : "memory");
                }
                float u[8];
#pragma unroll
                for (int c = kk + 1; c < 8; ++c) u[c] = round_h(__shfl_sync(0xffffffffu, a[kk & 3][c], src));
                if (lane == src) {
#pragma unroll
                    for (int c = kk + 1; c < 8; ++c) a[kk & 3][c] = u[c];
                }
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    if (r0 + r > t) {
#pragma unroll
                        for (int c = kk + 1; c < 8; ++c) a[r][c] = fmaf(-lv[r], u[c], a[r][c]);
                    }
            }
        }
    }
    if (!alive) bad = true;
    if (__syncthreads_or(bad)) {
        if (tid == 0) atomicOr(flag, 1);
        return;
    }
    // the factors (binary16) to A, U11 and L11^T (binary32, identity / zero padded to wp) to the stage
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int i = r0 + r;
        if (i < w && C0 < w) {
            S* dst = A + (int64_t)(K + i) * lda + K + C0;
            if (vec && C0 + 8 <= w) {
                store8(dst, a[r]);
            } else {
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    if (C0 + c < w) st_elem(dst + c, a[r][c]);
            }
        }
    }
    float* SU = stage;
    float* SL = stage + wp * wp;
    if (C0 < wp) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int i = r0 + r;
            if (i >= wp) continue;
            float uu[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int j = C0 + c;
                uu[c] = (i < w && j < w) ? ((j >= i) ? a[r][c] : 0.0f) : ((i == j) ? 1.0f : 0.0f);
            }
            *reinterpret_cast<float4*>(&SU[i * wp + C0]) = make_float4(uu[0], uu[1], uu[2], uu[3]);
            *reinterpret_cast<float4*>(&SU[i * wp + C0 + 4]) = make_float4(uu[4], uu[5], uu[6], uu[7]);
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int j = C0 + c;
            float ll[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int i = r0 + r;
                ll[r] = (i < w && j < w && i > j) ? a[r][c] : 0.0f;
            }
            if (r0 < wp) *reinterpret_cast<float4*>(&SL[j * wp + r0]) = make_float4(ll[0], ll[1], ll[2], ll[3]);
        }
    }
    if (tid < w) { ipiv[K + tid] = K + tid; PV[tid] = pvs[tid]; }
}




template <typename S>
__global__ void __launch_bounds__(kD16Threads, 1) k_diag_lu16(S* __restrict__ A, int64_t lda, int K, int w,
                                                             int* __restrict__ ipiv, int* __restrict__ flag,
                                                             float* __restrict__ stage)
{
    diag_lu16_body<false, S>(A, lda, K, w, ipiv, flag, stage);
}

// k_panel16: the diagonal block and the off-diagonal solves of one panel in
// one launch.  One CTA factors the diagonal block (the column pipeline above)
// and publishes every finished column t as {epoch, value} words; the other
// CTAs stream behind it, one step per published column:
//   row CTAs (256 rows of L21 each): row i at step t forms
//     x_it - sum_{k<t} l_ik u_kt (the sum in increasing k, one fused
//     multiply-add per term) from its own multipliers and U's column t, checks
//     it against the unrounded pivot and forms l_it = fl16(x / u_tt);
//   column CTAs (256 columns of U12 each): column j at step t forms
//     u_tj = fl16(a_tj - sum_{k<t} l_tk u_kj) from its own U entries and row t
//     of L11 (entry t of the published columns 0..t-1).
// Every entry takes the same fused multiply-adds in the same order as in the
// right-looking solves of k_offdiag16, so the results are bitwise those of
// k_diag_lu16 followed by k_offdiag16; only the schedule differs (the
// off-diagonal chains run one column behind the diagonal block instead of
// after it).  A published word is its own ready flag (the epoch is unique per
// launch and the buffer is cleared before each factorisation), so the
// producer needs no fence.  Each CTA keeps its rows' (columns') 128 values in
// shared memory; every wait is bounded and also gives up when the fast path
// has been abandoned.  The CTAs' roles follow the order they start in (see
// k_panel16), so no co-residency is needed.
constexpr int kPnlThreads = 512;
constexpr int kPnlRows = 256;   // at most this many rows (columns) per streaming CTA: one thread each
constexpr int kPnlFetchW = 14;  // warps 14 and 15 fetch the published columns (even / odd t)
constexpr int kPnlLd = 132;     // padded stride of the per-thread histories and the column cache (floats)
constexpr size_t kPnlSmem = (size_t)kPnlRows * kPnlLd * 4 + (size_t)128 * kPnlLd * 4 + 128 * 8;
constexpr long long kPnlSpin = 1LL << 22;

// Fetch warp: copy published column t (all 128 entries, lane l: entries 4l..4l+3)
// into the CTA's cache once its words carry this launch's epoch.  row_major:
// cache[e * kPnlLd + t] (row e of the panel, column t), else cache[t * kPnlLd + e].
__device__ __forceinline__ bool pnl_fetch(const unsigned long long* pub, int t, unsigned epoch, const int* flag,
                                          float* cache, bool row_major, const int* gave_up)
{
    const int lane = threadIdx.x & 31;
    const unsigned long long* q = pub + t * 128 + 4 * lane;
    for (long long it = 0; it < kPnlSpin; ++it) {
        unsigned long long v0, v1, v2, v3;
        asm volatile("ld.volatile.global.v2.u64 {%0, %1}, [%2];" : "=l"(v0), "=l"(v1) : "l"(q) : "memory");
        asm volatile("ld.volatile.global.v2.u64 {%0, %1}, [%2];" : "=l"(v2), "=l"(v3) : "l"(q + 2) : "memory");
        const bool ok = (unsigned)(v0 >> 32) == epoch && (unsigned)(v1 >> 32) == epoch &&
                        (unsigned)(v2 >> 32) == epoch && (unsigned)(v3 >> 32) == epoch;
        if (__all_sync(0xffffffffu, ok)) {
            const float f[4] = {__uint_as_float((unsigned)v0), __uint_as_float((unsigned)v1),
                                __uint_as_float((unsigned)v2), __uint_as_float((unsigned)v3)};
            if (row_major) {
#pragma unroll
                for (int r = 0; r < 4; ++r) cache[(4 * lane + r) * kPnlLd + t] = f[r];
            } else {
                *reinterpret_cast<float4*>(cache + t * kPnlLd + 4 * lane) = make_float4(f[0], f[1], f[2], f[3]);
            }
            return true;
        }
        if ((it & 63) == 63 && (*(volatile const int*)flag || *(volatile const int*)gave_up)) return false;
        __nanosleep(32);
    }
    return false;
}

__device__ __forceinline__ bool pnl_wait_ready(uint32_t bar, const int* gave_up)
{
    for (long long it = 0; it < kPnlSpin; ++it) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(bar)
                     : "memory");
        if (done) return true;
        if (*(volatile const int*)gave_up) return false;
    }
    return false;
}

// Steps t .. t+NB-1 of one streaming row (column) at once: each history
// value h[k], k < t, is loaded once for the NB dot products (shared-memory
// traffic / NB), then the NB x NB tail in order.  Every entry still takes its
// fused multiply-adds in increasing k.  c: the cache rows (ROWS: U's columns,
// else L11's rows), c + j * kPnlLd the one for step t + j.
template <bool ROWS, int NB>
__device__ __forceinline__ void pnl_steps(float* __restrict__ h, const float* __restrict__ c, int t, bool* bad)
{
    float acc[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) acc[j] = h[t + j];
    int k = 0;
#pragma unroll 4
    for (; k + 4 <= t; k += 4) {
        const float4 l4 = *reinterpret_cast<const float4*>(h + k);
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            const float4 c4 = *reinterpret_cast<const float4*>(c + j * kPnlLd + k);
            acc[j] = fmaf(-l4.x, c4.x, acc[j]);
            acc[j] = fmaf(-l4.y, c4.y, acc[j]);
            acc[j] = fmaf(-l4.z, c4.z, acc[j]);
            acc[j] = fmaf(-l4.w, c4.w, acc[j]);
        }
    }
    for (; k < t; ++k) {
        const float lk = h[k];
#pragma unroll
        for (int j = 0; j < NB; ++j) acc[j] = fmaf(-lk, c[j * kPnlLd + k], acc[j]);
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) {
#pragma unroll
        for (int jj = 0; jj < j; ++jj) acc[j] = fmaf(-h[t + jj], c[j * kPnlLd + t + jj], acc[j]);
        if (ROWS) {
            const float p = c[j * kPnlLd + t + j];
            const float ut = round_h(p);
            if (!(fabsf(acc[j]) <= fabsf(p))) *bad = true;
            h[t + j] = div_round_h(acc[j], ut, __frcp_rn(ut));
        } else {
            h[t + j] = round_h(acc[j]);
        }
    }
}

__device__ __forceinline__ bool pnl_test_ready(uint32_t bar)
{
    uint32_t done;
    asm volatile("{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done)
                 : "r"(bar)
                 : "memory");
    return done != 0;
}

// One streaming CTA: ROWS = rows of L21 (cache = U's columns, cache[t][k] = u_kt,
// entry t = the unrounded pivot), else columns of U12 (cache = L11 by rows,
// cache[t][k] = l_tk).  Threads 0..255 each own one row (column) and its
// 128-value history; warps 14 and 15 fetch the published columns; column t
// is signalled through ready[t] (an mbarrier per column, used once).
template <bool ROWS, typename S = __half>
__device__ __forceinline__ void panel16_stream(S* __restrict__ A, int64_t lda, int K, int w, int N, int blk,
                                               int rpc, __half* __restrict__ Ut, int ldut, int ut_col0, int ut_k0,
                                               int* __restrict__ flag, const unsigned long long* __restrict__ pub,
                                               unsigned epoch, unsigned* __restrict__ err)
{
    extern __shared__ __align__(16) float psm[];
    float* H = psm;                          // H[r * kPnlLd + t]: a, replaced by l (rows) / u (columns) at step t
    float* Cc = psm + kPnlRows * kPnlLd;     // the published columns
    uint64_t* ready = reinterpret_cast<uint64_t*>(Cc + 128 * kPnlLd);
    __shared__ int gave_up;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int idx = K + w + blk * rpc + tid;  // row (ROWS) or column of this thread
    const bool mine = tid < rpc, live = mine && idx < N;
    float* h = H + (mine ? tid : 0) * kPnlLd;
    if (tid == 0) gave_up = 0;
    if (tid < 128) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((unsigned)__cvta_generic_to_shared(&ready[tid])));
    const bool vec = (w % 8 == 0) && (lda % 8 == 0) && ((((uintptr_t)(A + K)) & 15) == 0);
    if (live) {
        if (ROWS) {
            const S* R = A + (int64_t)idx * lda + K;
            if (vec) {
                for (int t = 0; t < w; t += 8) load8(R + t, h + t);
            } else {
                for (int t = 0; t < w; ++t) h[t] = ld_elem(R + t);
            }
        } else {
            for (int t = 0; t < w; ++t) h[t] = ld_elem(A + (int64_t)(K + t) * lda + idx);
        }
    }
    __syncthreads();
    bool bad = false;
    if (warp >= kPnlFetchW) {
        // fetchers: warp 14 the even columns, warp 15 the odd ones
        const int f = warp - kPnlFetchW;
        const int tmax = ROWS ? w : w - 1;  // the column CTAs never need the last column
        for (int t = f; t < tmax; t += 2) {
            if (!pnl_fetch(pub, t, epoch, flag, Cc, !ROWS, &gave_up)) {
                *(volatile int*)&gave_up = 1;
                break;
            }
            __syncwarp();
            if ((tid & 31) == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"((unsigned)__cvta_generic_to_shared(&ready[t]))
                             : "memory");
        }
    } else if (mine) {
        // rows need columns t..t+nb-1; columns need L11's rows t..t+nb-1, i.e. columns up to t+nb-2
        const int lag = ROWS ? 0 : 1;
        auto bar_of = [&](int col) { return (unsigned)__cvta_generic_to_shared(&ready[col]); };
        for (int t = 0; t < w;) {
            const int need = t - lag;
            if (need >= 0 && !pnl_wait_ready(bar_of(need), &gave_up)) {
                *(volatile int*)&gave_up = 1;
                break;
            }
            // take up to four steps when their columns are already in (decided once per warp)
            int nb = 1;
            if ((threadIdx.x & 31) == 0)
                while (nb < 4 && t + nb < w && (need + nb < 0 || pnl_test_ready(bar_of(need + nb)))) ++nb;
            nb = __shfl_sync(0xffffffffu, nb, 0);
            __syncwarp();  // lane 0's acquire of the extra columns orders the whole warp's reads
            if (live) {
                const float* c = Cc + t * kPnlLd;
                switch (nb) {
                case 4: pnl_steps<ROWS, 4>(h, c, t, &bad); break;
                case 3: pnl_steps<ROWS, 3>(h, c, t, &bad); break;
                case 2: pnl_steps<ROWS, 2>(h, c, t, &bad); break;
                default: pnl_steps<ROWS, 1>(h, c, t, &bad); break;
                }
            }
            t += nb;
        }
    }
    if (__syncthreads_or(bad) && tid == 0) atomicOr(flag, 1);
    if (gave_up) {
        if (tid == 0) {
            // a timeout (not an abandoned fast path) is an error; either way the
            // caller refactors with interchanges
            if (!*(volatile const int*)flag) atomicOr(err, (unsigned)ERR_TIMEOUT_OTHER);
            atomicOr(flag, 1);
        }
        return;
    }
    if (!live) return;
    if (ROWS) {
        S* R = A + (int64_t)idx * lda + K;
        if (vec) {
            for (int t = 0; t < w; t += 8) store8(R + t, h + t);
        } else {
            for (int t = 0; t < w; ++t) st_elem(R + t, h[t]);
        }
    } else {
        for (int t = 0; t < w; ++t) st_elem(A + (int64_t)(K + t) * lda + idx, h[t]);
        // U12^T for the tensor-core update: row idx - ut_col0, columns ut_k0 .. ut_k0 + w - 1
        // (columns left of ut_col0 are not part of that update)
        if (Ut && idx >= ut_col0) {
            __half* u0 = Ut + (int64_t)(idx - ut_col0) * ldut + ut_k0;
            if ((w % 8 == 0) && (ldut % 8 == 0) && (ut_k0 % 8 == 0) && ((((uintptr_t)Ut) & 15) == 0)) {
                for (int t = 0; t < w; t += 8) {
                    __align__(16) __half e[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) e[q] = __float2half_rn(h[t + q]);
                    *reinterpret_cast<uint4*>(u0 + t) = *reinterpret_cast<const uint4*>(e);
                }
            } else {
                for (int t = 0; t < w; ++t) u0[t] = __float2half_rn(h[t]);
            }
        }
    }
}

// S: the storage the panel is read from and written to: the binary16 matrix,
// or (two-level LU) its single-precision shadow over the current outer block.
// Ut: U12^T in binary16 for the columns from ut_col0 (at K offset ut_k0).
// Roles are handed out in the order the CTAs start (an atomic ticket; panel p
// of a factorisation counts in word p % 2, its first CTA clears the other word
// and its last one its own; both are cleared when the factorisation starts): ticket 0
// factors the diagonal block and publishes its columns, tickets 1..nrb stream
// rows, the rest stream columns.  A CTA only ever waits on the diagonal CTA,
// which took its ticket before any waiting CTA existed and so is running: the
// launch needs no co-residency.
template <typename S>
__global__ void __launch_bounds__(kPnlThreads, 1) k_panel16(S* __restrict__ A, int64_t lda, int K, int w, int N,
                                                           int nrb, int rpc, int* __restrict__ ipiv, int* __restrict__ flag,
                                                           float* __restrict__ stage, __half* __restrict__ Ut,
                                                           int ldut, int ut_col0, int ut_k0,
                                                           unsigned long long* __restrict__ pub, unsigned epoch,
                                                           unsigned* __restrict__ err, int* __restrict__ tickets,
                                                           int slot)
{
    __shared__ int role;
    if (threadIdx.x == 0) {
        const int t = atomicAdd(&tickets[slot], 1);
        if (t == 0) tickets[slot ^ 1] = 0;                // for the next panel (launched after this one ends)
        if (t == (int)gridDim.x - 1) tickets[slot] = 0;  // every ticket is taken: this launch's word is free
        role = t;
    }
    __syncthreads();
    const int r = role;
    if (r == 0)
        diag_lu16_body<true, S>(A, lda, K, w, ipiv, flag, stage, pub, epoch);
    else if (r <= nrb)
        panel16_stream<true, S>(A, lda, K, w, N, r - 1, rpc, Ut, ldut, ut_col0, ut_k0, flag, pub, epoch, err);
    else
        panel16_stream<false, S>(A, lda, K, w, N, r - 1 - nrb, rpc, Ut, ldut, ut_col0, ut_k0, flag, pub, epoch, err);
}

// k_offdiag16: L21 = A21 U11^{-1} (row role) and U12 = L11^{-1} A12 (column
// role) for a panel of width w, one thread per row (or column), 128 per CTA.
// A thread takes its row in 32-wide chunks: the chunk is first updated with
// the row's multipliers of the earlier chunks (kept in shared memory, one
// column of X per thread), then solved against the chunk's diagonal 32 x 32
// block of U11: at step t the thread checks its pre-division value against
// the unrounded pivot, forms l = fl16(x_t / u_tt) and updates the rest of
// the chunk.  The column role is the same with L11 and no division (U
// entries rounded to binary16 as they are formed), and also writes U12^T for
// the tensor-core update.  U11 / L11^T come from the stage as binary32 (exact
// binary16 values) and are read by all threads at once (broadcast).  Every
// entry takes its updates in increasing t, as in right-looking elimination;
// with no shuffles or group hand-offs the per-step chain is one multiplier
// formation and one fused multiply-add.
constexpr int kO16Threads = 128;
constexpr int kO16Rows = 128;  // rows or columns per CTA

// R: rows (columns) per CTA, one thread each: 128, or 256 for wide launches of
// 128-column panels (twice the warps per SM at one CTA per SM)
__host__ __device__ size_t offdiag16_smem(int wp, int R = kO16Rows)
{
    return ((size_t)wp * wp + (size_t)wp * R + 2 * wp) * sizeof(float);
}

template <typename S = __half, int ROWS = kO16Rows>
__device__ __forceinline__ void offdiag16_body(S* __restrict__ A, int64_t lda, int K, int w, int N,
                                               int nrow_blocks, __half* __restrict__ Ut, int ldut,
                                               int* __restrict__ flag, const float* stage, int bid,
                                               int ut_col0 = -1, int ut_k0 = 0, int tid_in = -1,
                                               float* smem = nullptr, int off0 = 0)
{
    if (ut_col0 < 0) ut_col0 = K + w;
    if (tid_in < 0 && *(volatile int*)flag) return;  // (a group of a larger CTA: its caller checked)
    extern __shared__ __align__(16) float osm[];
    const int wp = (w + 31) & ~31, nc = wp / 32;
    // tid_in / smem: a group of 128 threads of a larger CTA and its own shared region (the
    // persistent grouped factorisation runs four such groups side by side)
    float* D = smem ? smem : osm;    // U11 (row role) or L11^T (column role), wp x wp
    float* X = D + wp * wp;          // X[t * ROWS + tid]: this thread's multipliers / U entries
    float* pv = X + wp * ROWS;          // |a_tt|, unrounded
    float* rinv = pv + wp;           // 1 / u_tt, correctly rounded
    const int tid = tid_in >= 0 ? tid_in : (int)threadIdx.x;
    const bool row_role = bid < nrow_blocks;
    {
        const float4* s4 = reinterpret_cast<const float4*>(stage + (row_role ? 0 : wp * wp));
        float4* d4 = reinterpret_cast<float4*>(D);
        const int nv = wp * wp / 4;
#pragma unroll 4
        for (int v = tid; v < nv; v += ROWS) d4[v] = s4[v];
        if (tid < wp) pv[tid] = fabsf(stage[kStagePivOff + tid]);
    }
    __syncthreads();
    if (row_role && tid < wp) rinv[tid] = __frcp_rn(D[tid * wp + tid]);
    __syncthreads();
    // off0: the first off0 rows (columns) below (right of) the block are someone else's
    const int idx = K + w + off0 + (row_role ? bid : bid - nrow_blocks) * ROWS + tid;
    const bool live = idx < N;
    float* Xt = X + tid;
    if (row_role) {
        bool bad = false;
        S* R = A + (int64_t)min(idx, N - 1) * lda + K;
        const bool vec = (w % 32 == 0) && ((((uintptr_t)(A + K)) & 15) == 0) && (lda % 8 == 0);
        for (int c = 0; c < nc; ++c) {
            const int j0 = 32 * c;
            float x[32];
            if (vec && live) {
#pragma unroll
                for (int q = 0; q < 4; ++q) load8(R + j0 + 8 * q, x + 8 * q);
            } else {
#pragma unroll
                for (int k = 0; k < 32; ++k) x[k] = (live && j0 + k < w) ? ld_elem(R + j0 + k) : 0.0f;
            }
#pragma unroll 8
            for (int t = 0; t < j0; ++t) {
                const float l = Xt[t * ROWS];
                const float4* Dt = reinterpret_cast<const float4*>(D + t * wp + j0);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float4 d = Dt[q];
                    x[4 * q + 0] = fmaf(-l, d.x, x[4 * q + 0]);
                    x[4 * q + 1] = fmaf(-l, d.y, x[4 * q + 1]);
                    x[4 * q + 2] = fmaf(-l, d.z, x[4 * q + 2]);
                    x[4 * q + 3] = fmaf(-l, d.w, x[4 * q + 3]);
                }
            }
#pragma unroll
            for (int tt = 0; tt < 32; ++tt) {
                const int t = j0 + tt;
                const float* Dt = D + t * wp + j0;
                if (live && t < w && !(fabsf(x[tt]) <= pv[t])) bad = true;
                const float l = div_round_h(x[tt], Dt[tt], rinv[t]);
                x[tt] = l;
#pragma unroll
                for (int k = tt + 1; k < 32; ++k) x[k] = fmaf(-l, Dt[k], x[k]);
            }
            // the chunk's multipliers for the later chunks (no shared-memory stores inside
            // the solve, so the loads of U11 can move ahead of the division chain)
#pragma unroll
            for (int tt = 0; tt < 32; ++tt) Xt[(j0 + tt) * ROWS] = x[tt];
            if (live) {
                if (vec) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) store8(R + j0 + 8 * q, x + 8 * q);
                } else {
#pragma unroll
                    for (int k = 0; k < 32; ++k)
                        if (j0 + k < w) st_elem(R + j0 + k, x[k]);
                }
            }
        }
        if (__syncthreads_or(bad) && tid == 0) atomicOr(flag, 1);
    } else {
        const int col = min(idx, N - 1);
        for (int c = 0; c < nc; ++c) {
            const int k0 = 32 * c;
            float x[32];
#pragma unroll
            for (int k = 0; k < 32; ++k)
                x[k] = (live && k0 + k < w) ? ld_elem(A + (int64_t)(K + k0 + k) * lda + col) : 0.0f;
#pragma unroll 8
            for (int t = 0; t < k0; ++t) {
                const float u = Xt[t * ROWS];
                const float4* Dt = reinterpret_cast<const float4*>(D + t * wp + k0);  // L[k0 + k][t]
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float4 d = Dt[q];
                    x[4 * q + 0] = fmaf(-d.x, u, x[4 * q + 0]);
                    x[4 * q + 1] = fmaf(-d.y, u, x[4 * q + 1]);
                    x[4 * q + 2] = fmaf(-d.z, u, x[4 * q + 2]);
                    x[4 * q + 3] = fmaf(-d.w, u, x[4 * q + 3]);
                }
            }
#pragma unroll
            for (int tt = 0; tt < 32; ++tt) {
                const int t = k0 + tt;
                const float* Dt = D + t * wp + k0;
                const float u = round_h(x[tt]);
                x[tt] = u;
#pragma unroll
                for (int k = tt + 1; k < 32; ++k) x[k] = fmaf(-Dt[k], u, x[k]);
            }
#pragma unroll
            for (int tt = 0; tt < 32; ++tt) Xt[(k0 + tt) * ROWS] = x[tt];
            if (live) {
#pragma unroll
                for (int k = 0; k < 32; ++k)
                    if (k0 + k < w) st_elem(A + (int64_t)(K + k0 + k) * lda + col, x[k]);
                if (Ut && idx >= ut_col0) {
                    // U12^T row (the tensor-core B operand): 32 consecutive entries
                    __half* u0 = Ut + (int64_t)(idx - ut_col0) * ldut + ut_k0 + k0;
                    if (k0 + 32 <= w && (ldut % 8 == 0) && (ut_k0 % 8 == 0) && ((((uintptr_t)Ut) & 15) == 0)) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            __align__(16) __half h[8];
#pragma unroll
                            for (int k = 0; k < 8; ++k) h[k] = __float2half_rn(x[8 * q + k]);
                            reinterpret_cast<uint4*>(u0)[q] = *reinterpret_cast<const uint4*>(h);
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < 32; ++k)
                            if (k0 + k < w) u0[k] = __float2half_rn(x[k]);
                    }
                }
            }
        }
    }
}

template <typename S, int ROWS = kO16Rows>
__global__ void __launch_bounds__(ROWS) k_offdiag16(S* __restrict__ A, int64_t lda, int K, int w, int N,
                                                 int nrow_blocks, __half* __restrict__ Ut, int ldut,
                                                 int* __restrict__ flag, const float* __restrict__ stage,
                                                 int ut_col0, int ut_k0, int off0)
{
    offdiag16_body<S, ROWS>(A, lda, K, w, N, nrow_blocks, Ut, ldut, flag, stage, (int)blockIdx.x, ut_col0, ut_k0, -1,
                            nullptr, off0);
}

// The off-diagonal solves of one panel: 128 rows (columns) per CTA, or 256 for a
// panel of 128 columns whose 128-row CTAs would not all fit at once (one CTA per
// SM either way at that width, so twice the warps per SM).  Bitwise the same
// results: every row (column) is solved by one thread in the same order.
template <typename S>
static nl_status launch_offdiag16(S* A, int64_t ld, int K, int wd, int N, __half* ut, int ldut, int* flag,
                                  const float* stage, int ut_col0, int ut_k0, cudaStream_t st, int off0 = 0)
{
    const int rest = N - K - wd - off0, wp = (int)round_up(wd, 32);  // rows (columns) from K + wd + off0
    const bool wide = wp > 64 && 2 * (int)cdiv(rest, kO16Rows) > num_sms();
    prof_begin("k_offdiag16", st);
    if (wide) {
        const int nrb = (int)cdiv(rest, 256);
        k_offdiag16<S, 256><<<2 * nrb, 256, offdiag16_smem(wp, 256), st>>>(A, ld, K, wd, N, nrb, ut, ldut, flag, stage,
                                                                         ut_col0, ut_k0, off0);
    } else {
        const int nrb = (int)cdiv(rest, kO16Rows);
        k_offdiag16<S><<<2 * nrb, kO16Threads, offdiag16_smem(wp), st>>>(A, ld, K, wd, N, nrb, ut, ldut, flag, stage,
                                                                        ut_col0, ut_k0, off0);
    }
    prof_end("k_offdiag16", st);
    NL_CUDA_OK(cudaGetLastError());
    return NL_OK;
}

// C <- C - A B with per-element sequential fused multiply-adds over k in
// order, accumulated in T and stored once (rounded to binary16 for __half).
template <typename S, typename T>
__device__ __forceinline__ void gemm_simt_body(int M, int Nc, int K, const S* __restrict__ A, int64_t lda,
                                                   const S* __restrict__ B, int64_t ldb, S* __restrict__ C,
                                                   int64_t ldc, const int* __restrict__ flag, int m0, int n0)
{
    if (flag && *(volatile const int*)flag) return;
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            int i = m0 + ty + 16 * a, j = n0 + tx + 16 * b;
            acc[a][b] = (i < M && j < Nc) ? (T)ld_elem(C + (int64_t)i * ldc + j) : T(0);
        }
    for (int k0 = 0; k0 < K; k0 += BK) {
        __syncthreads();
        for (int q = threadIdx.x; q < BM * BK; q += 256) {
            int r = q / BK, kk = q % BK;
            int i = m0 + r, k = k0 + kk;
            As[kk][r] = (i < M && k < K) ? (T)ld_elem(A + (int64_t)i * lda + k) : T(0);
        }
        for (int q = threadIdx.x; q < BK * BN; q += 256) {
            int kk = q / BN, x = q % BN;
            int k = k0 + kk, j = n0 + x;
            Bs[kk][x] = (k < K && j < Nc) ? (T)ld_elem(B + (int64_t)k * ldb + j) : T(0);
        }
        __syncthreads();
        const int kmax = min(BK, K - k0);
        for (int kk = 0; kk < kmax; ++kk) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(-av[a], bv[b], acc[a][b]);
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            int i = m0 + ty + 16 * a, j = n0 + tx + 16 * b;
            if (i < M && j < Nc) st_elem(C + (int64_t)i * ldc + j, acc[a][b]);
        }
}

template <typename S, typename T>
__global__ void __launch_bounds__(256) k_gemm_simt(int M, int Nc, int K, const S* __restrict__ A, int64_t lda,
                                                   const S* __restrict__ B, int64_t ldb, S* __restrict__ C,
                                                   int64_t ldc, const int* __restrict__ flag)
{
    gemm_simt_body<S, T>(M, Nc, K, A, lda, B, ldb, C, ldc, flag, (int)blockIdx.y * 64, (int)blockIdx.x * 64);
}

// ------------------------------------------------------------------ host --

// Workspace layout: the interchanging path's working panel (N x min(nb, 128)),
// U12^T for the tensor-core update (N x nb binary16), info/flag words, the
// diagonal-block stage, the published columns, and for an outer block above
// 128 (two-level LU, binary16 only) the single-precision shadow N x ld, else
// (binary16) the look-ahead's second U12^T buffer.
size_t lu_work_bytes(int N, int nb, bool fp64)
{
    size_t el = fp64 ? 8 : 4;
    size_t pnl = (size_t)N * std::min(nb, 128) * el;
    size_t ut = fp64 ? 0 : (size_t)round_up(N, 128) * nb * 2;
    size_t shadow = fp64 ? 0 : (nb > 128 ? (size_t)N * round_up(N, 64) * 4 + 256 : round_up(ut, 256));
    return round_up(pnl, 256) + round_up(ut, 256) + 256 + (size_t)2 * 128 * 128 * 8 + 128 * 8 +
           round_up((size_t)128 * 128 * 8, 256) + shadow;
}

void lu_work_carve(void* base, int N, int nb, bool fp64, LuWork* w)
{
    char* p = (char*)base;
    size_t el = fp64 ? 8 : 4;
    w->pnl = p;
    p += round_up((size_t)N * std::min(nb, 128) * el, 256);
    size_t ut = fp64 ? 0 : (size_t)round_up(N, 128) * nb * 2;
    w->ut = fp64 ? nullptr : (__half*)p;
    p += round_up(ut, 256);
    w->info = (int*)p;
    w->flag = w->info + 1;
    p += 256;
    w->stage = p;
    p += (size_t)2 * 128 * 128 * 8 + 128 * 8;
    w->pub = (unsigned long long*)p;
    p += round_up((size_t)128 * 128 * 8, 256);
    w->ut2 = nullptr;
    if (!fp64 && nb > 128) {
        w->p32 = (float*)p;
        w->ldp32 = round_up(N, 64);
    } else {
        w->p32 = nullptr;
        w->ldp32 = 0;
        if (!fp64) w->ut2 = (__half*)p;
    }
}

nl_status lu_side_prepare(LuWork* w, cudaStream_t st)
{
    // one step below st's priority (lower priority = larger number): the rest of an update has
    // a panel's time of slack, so it yields SMs to the latency-bound panels of concurrent solves
    int prio = 0, least = 0, greatest = 0;
    NL_CUDA_OK(cudaStreamGetPriority(st, &prio));
    NL_CUDA_OK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    prio = std::min(prio + 1, least);
    if (w->side) {
        int have = 0;
        NL_CUDA_OK(cudaStreamGetPriority(w->side, &have));
        if (have == prio) return NL_OK;
        NL_CUDA_OK(cudaStreamSynchronize(w->side));
        NL_CUDA_OK(cudaStreamDestroy(w->side));
        w->side = nullptr;
    }
    NL_CUDA_OK(cudaStreamCreateWithPriority(&w->side, cudaStreamNonBlocking, prio));
    if (!w->ev_fork) NL_CUDA_OK(cudaEventCreateWithFlags(&w->ev_fork, cudaEventDisableTiming));
    for (auto& e : w->ev_join)
        if (!e) NL_CUDA_OK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return NL_OK;
}

void lu_side_release(LuWork* w)
{
    if (w->side) cudaStreamDestroy(w->side);
    if (w->ev_fork) cudaEventDestroy(w->ev_fork);
    for (auto& e : w->ev_join)
        if (e) cudaEventDestroy(e);
    w->side = nullptr;
    w->ev_fork = w->ev_join[0] = w->ev_join[1] = nullptr;
}

template <typename T, int NBL, int R, bool RND>
static nl_status launch_leaf_r(T* P, int ldp, int k0, int M, int w, int wl, int* ipiv_out, int piv_base, int* info,
                               int C, int rows_per_cta, cudaStream_t st)
{
    auto kern = k_leaf<T, NBL, R, RND>;
    if (C > 1) {
        static bool attr_done = false;
        if (!attr_done) {
            NL_CUDA_OK(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
            attr_done = true;
        }
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(C);
        cfg.blockDim = dim3(kLeafThreads);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = st;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        NL_CUDA_OK(cudaLaunchKernelEx(&cfg, kern, P, ldp, k0, M, w, wl, ipiv_out, piv_base, info, C, rows_per_cta));
    } else {
        kern<<<1, kLeafThreads, 0, st>>>(P, ldp, k0, M, w, wl, ipiv_out, piv_base, info, 1, rows_per_cta);
        NL_CUDA_OK(cudaGetLastError());
    }
    return NL_OK;
}

// Cluster size and rows per thread for a leaf of Ml rows: the fewest CTAs
// (cheapest exchange) with at most 4 (8 beyond 16384 rows) rows per thread.
template <typename T, int NBL, bool RND>
static nl_status launch_leaf(T* P, int ldp, int k0, int M, int w, int wl, int* ipiv_out, int piv_base, int* info,
                             cudaStream_t st)
{
    const int Ml = M - k0;
    // at most 4 rows per thread (spill-free) unless the leaf needs more than
    // 16 CTAs at that density
    int C = (int)cdiv(Ml, 4 * kLeafThreads);
    if (C > kMaxCluster) C = (int)cdiv(Ml, 8 * kLeafThreads);
    if (C > kMaxCluster) {
        set_error("LU leaf: %d rows exceed the register-resident limit", Ml);
        return NL_EINVAL;
    }
    if (C > 8) C = 16;
    else if (C > 4) C = 8;
    else if (C > 2) C = 4;
    const int rows_per_cta = (int)cdiv(Ml, C);
    const int R = (int)cdiv(rows_per_cta, kLeafThreads);
    if (R <= 1) return launch_leaf_r<T, NBL, 1, RND>(P, ldp, k0, M, w, wl, ipiv_out, piv_base, info, C, rows_per_cta, st);
    if (R <= 2) return launch_leaf_r<T, NBL, 2, RND>(P, ldp, k0, M, w, wl, ipiv_out, piv_base, info, C, rows_per_cta, st);
    if (R <= 4) return launch_leaf_r<T, NBL, 4, RND>(P, ldp, k0, M, w, wl, ipiv_out, piv_base, info, C, rows_per_cta, st);
    return launch_leaf_r<T, NBL, 8, RND>(P, ldp, k0, M, w, wl, ipiv_out, piv_base, info, C, rows_per_cta, st);
}

template <typename S, typename T>
static nl_status launch_gemm_simt(int M, int Nc, int K, const S* A, int64_t lda, const S* B, int64_t ldb, S* C,
                                  int64_t ldc, cudaStream_t st, const int* flag = nullptr)
{
    if (M <= 0 || Nc <= 0 || K <= 0) return NL_OK;
    dim3 grid((unsigned)cdiv(Nc, 64), (unsigned)cdiv(M, 64));
    k_gemm_simt<S, T><<<grid, 256, 0, st>>>(M, Nc, K, A, lda, B, ldb, C, ldc, flag);
    NL_CUDA_OK(cudaGetLastError());
    return NL_OK;
}

__global__ void k_transpose16(int R, int Cc, const __half* __restrict__ in, int64_t ldi, __half* __restrict__ out,
                              int64_t ldo)
{
    __shared__ __half tile[32][33];
    int c = blockIdx.x * 32 + threadIdx.x, r = blockIdx.y * 32 + threadIdx.y;
    for (int k = 0; k < 32; k += 8)
        if (r + k < R && c < Cc) tile[threadIdx.y + k][threadIdx.x] = in[(int64_t)(r + k) * ldi + c];
    __syncthreads();
    c = blockIdx.y * 32 + threadIdx.x;
    r = blockIdx.x * 32 + threadIdx.y;
    for (int k = 0; k < 32; k += 8)
        if (r + k < Cc && c < R) out[(int64_t)(r + k) * ldo + c] = tile[threadIdx.x][threadIdx.y + k];
}

nl_status launch_transpose16(int R, int Cc, const __half* in, int64_t ldi, __half* out, int64_t ldo, cudaStream_t st)
{
    dim3 grid((unsigned)cdiv(Cc, 32), (unsigned)cdiv(R, 32));
    k_transpose16<<<grid, dim3(32, 8), 0, st>>>(R, Cc, in, ldi, out, ldo);
    NL_CUDA_OK(cudaGetLastError());
    return NL_OK;
}

nl_status gemm16_update(int M, int Nc, int K, const __half* A, int64_t lda, const __half* B, int64_t ldb, __half* C,
                        int64_t ldc, int gemm, cudaStream_t st)
{
    if (gemm == 2 || gemm == 3) {
        // the tensor-core path takes B transposed (K-major): build it
        __half* Bt = nullptr;
        NL_CUDA_OK(cudaMallocAsync((void**)&Bt, (size_t)round_up(Nc, 128) * K * 2, st));
        nl_status s = launch_transpose16(K, Nc, B, ldb, Bt, K, st);
        if (s == NL_OK) s = tc_gemm16_update(M, Nc, K, A, lda, Bt, K, C, ldc, st, nullptr, gemm == 3);
        cudaFreeAsync(Bt, st);
        return s;
    }
    return launch_gemm_simt<__half, float>(M, Nc, K, A, lda, B, ldb, C, ldc, st);
}

// A22 <- A22 - L21 U12 for the panel [K, K+wd): tcgen05 when possible.
template <typename T, typename S>
static nl_status trailing_update(int N, S* A, int64_t ld, int K, int wd, int nb, bool tc, const __half* ut,
                                 const int* flag, cudaStream_t st)
{
    const int rest = N - K - wd;
    S* L21 = A + (int64_t)(K + wd) * ld + K;
    S* U12 = A + (int64_t)K * ld + K + wd;
    S* A22 = A + (int64_t)(K + wd) * ld + K + wd;
    if (tc) {
        if constexpr (std::is_same<S, __half>::value) return tc_gemm16_update(rest, rest, wd, L21, ld, ut, nb, A22, ld, st, flag);
    }
    return launch_gemm_simt<S, T>(rest, rest, wd, L21, ld, U12, ld, A22, ld, st, flag);
}

// The streaming panel (k_panel16): one CTA for the diagonal block plus
// ceil(rest / rpc) CTAs for the rows of L21 and as many for the columns of
// U12 (rpc = 128 while they all fit on the device at once, else 256), when
// they fit in one wave; otherwise the two-launch path.
static int panel16_max_ctas()
{
    // computed once; concurrent first callers compute the same value (never a transient 0)
    static std::atomic<int> cap{-1};
    int c = cap.load(std::memory_order_acquire);
    if (c < 0) {
        c = 0;
        int dev = 0, nsm = 0, per = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            set_max_dynamic_smem((const void*)k_panel16<__half>) == NL_OK &&
            set_max_dynamic_smem((const void*)k_panel16<float>) == NL_OK &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_panel16<__half>, kPnlThreads, kPnlSmem) == cudaSuccess)
            c = per * nsm;
        cudaGetLastError();
        cap.store(c, std::memory_order_release);
    }
    return c;
}

// Rows (columns) per streaming CTA: 128 when the launch then fits on the GPU
// (with 256 the full CTAs fall behind the diagonal block; 64 is no faster and
// takes twice the SMs from concurrent solves), else 256; 0 when neither fits
// (two launches instead).
static int panel16_rows_per_cta(int rest, int pref = 0)
{
    // 128 rows per CTA while every CTA fits at once (more CTAs in the chain's shadow), else
    // 256; beyond what fits in one wave the two launches are as fast (measured on GB300 at
    // N = 32768: the factorisation takes 65-66 ms either way)
    const int cap = panel16_max_ctas();
    for (int rpc : {pref == kPnlRows ? kPnlRows : 128, kPnlRows})
        if (1 + 2 * (int)cdiv(rest, rpc) <= cap) return rpc;
    return 0;
}

// Rows (and columns) of a panel the streaming launch takes: all of them when its
// CTAs fit on the device at once, else as many as 256-row CTAs fitting at once
// cover (the rest go to a following off-diagonal launch); 0 = none.
static int panel16_fit_rows(int rest, int pref = 0)
{
    if (panel16_rows_per_cta(rest, pref) > 0) return rest;
    const int nrb = (panel16_max_ctas() - 1) / 2;
    return nrb >= 1 ? std::min(rest, nrb * kPnlRows) : 0;
}

static std::atomic<unsigned> g_panel_epoch{0};

template <typename S>
static nl_status launch_panel16(S* A, int64_t ld, int K, int wd, int N, int* ipiv, const LuWork& w, __half* Ut,
                                int ldut, cudaStream_t st, int slot, int ut_col0 = -1, int ut_k0 = 0)
{
    if (ut_col0 < 0) ut_col0 = K + wd;
    const int rest = N - K - wd;
    int rpc = panel16_rows_per_cta(rest, w.stream);
    int nrb = (int)cdiv(rest, rpc);
    unsigned epoch = ++g_panel_epoch;
    if (epoch == 0) epoch = ++g_panel_epoch;  // 0 is the cleared buffer's tag
    int* flag = w.flag;
    float* stage = (float*)w.stage;
    unsigned long long* pub = w.pub;
    unsigned* err = tc_error_word();
    if (!err) err = (unsigned*)(w.info + 2);  // (a word of the info block nobody else uses)
    int* tickets = w.info + 8;  // two counters (+8, +9) of the info block; slot: the panel's index mod 2
    prof_begin("k_panel16", st);
    k_panel16<S><<<1 + 2 * nrb, kPnlThreads, kPnlSmem, st>>>(A, ld, K, wd, N, nrb, rpc, ipiv, flag, stage, Ut, ldut,
                                                            ut_col0, ut_k0, pub, epoch, err, tickets, slot);
    prof_end("k_panel16", st);
    NL_CUDA_OK(cudaGetLastError());
    return NL_OK;
}

template <typename T, typename S, int NBL, bool RND>
static nl_status lu_factor_impl(int N, S* A, int64_t ld, int* ipiv, int nb, int gemm, bool fast, const LuWork& w,
                                cudaStream_t st, int* launches)
{
    T* P = (T*)w.pnl;
    const int ldp = nb;
    int nl = 0;
    NL_CUDA_OK(cudaMemsetAsync(w.info, 0, 10 * sizeof(int), st));  // info, flag, ..., the panel's role ticket
    constexpr bool kHalf = std::is_same<S, __half>::value;
    static bool smem_set = false;
    if (!smem_set) {
        if (set_max_dynamic_smem((const void*)k_trsm_u12<T, S, RND>) != NL_OK) return NL_ECUDA;
        if constexpr (kHalf) {
            if (set_max_dynamic_smem((const void*)k_offdiag16<__half>) != NL_OK ||
                set_max_dynamic_smem((const void*)k_offdiag16<float>) != NL_OK ||
                set_max_dynamic_smem((const void*)k_offdiag16<__half, 256>) != NL_OK ||
                set_max_dynamic_smem((const void*)k_offdiag16<float, 256>) != NL_OK ||
                set_max_dynamic_smem((const void*)k_diag_lu16<__half>) != NL_OK ||
                set_max_dynamic_smem((const void*)k_diag_lu16<float>) != NL_OK)
                return NL_ECUDA;
        } else {
            if (set_max_dynamic_smem((const void*)k_offdiag<T, S, RND>) != NL_OK ||
                set_max_dynamic_smem((const void*)k_diag_lu<T, S, RND>) != NL_OK)
                return NL_ECUDA;
        }
        smem_set = true;
    }
    bool pub_cleared = false;
    // Look-ahead (fast path, tensor-core update): the update after panel q is split into the
    // cross (the first 128-row and 128-column tile strips of the trailing matrix, which hold
    // panel q + 1), one launch on st, and the rest on w.side, which then runs in the shadow of
    // panel q + 1 and is joined back (ev_join[q % 2]) before the cross of update q + 1.  The
    // tiles are the same tcgen05 tiles as in one update, so the factors are bitwise the same.
    // Panels alternate U12^T buffers.
    constexpr int kLaTile = 128;  // the tcgen05 update's tile (M = N = 128)
    const bool la = kHalf && fast && gemm == 2 && nb <= kLaTile && w.side && w.ut2 && w.ev_fork && w.ev_join[0] &&
                    w.ev_join[1];
    struct Join {
        const LuWork& w;
        cudaStream_t st;
        int pending = 0;  // bit q % 2: the rest of update q is recorded on ev_join[q % 2], not yet joined
        bool wait(int q)
        {
            if (q < 0 || !((pending >> (q & 1)) & 1)) return true;
            pending &= ~(1 << (q & 1));
            return cudaStreamWaitEvent(st, w.ev_join[q & 1], 0) == cudaSuccess;
        }
        bool all() { return wait(0) && wait(1); }
        ~Join() { all(); }
    } join{w, st};
    auto join_ok = [&](bool ok) -> nl_status {
        if (ok) return NL_OK;
        set_error("LU look-ahead: cudaStreamWaitEvent failed");
        return NL_ECUDA;
    };
    auto ut_of = [&](int K) { return (la && ((K / nb) & 1)) ? w.ut2 : w.ut; };
    // the update after the panel at K (width wd)
    auto update = [&](int K, int wd, bool tc, const __half* utp) -> nl_status {
        const int rest = N - K - wd, q = K / nb;
        if (!(la && tc)) {
            NL_TRY(join_ok(join.all()));
            return trailing_update<T, S>(N, A, ld, K, wd, nb, tc, utp, w.flag, st);
        }
        if constexpr (kHalf) {
            S* L21 = A + (int64_t)(K + wd) * ld + K;
            S* A22 = A + (int64_t)(K + wd) * ld + K + wd;
            const bool side_now = rest > kLaTile;
            if (side_now) NL_CUDA_OK(cudaEventRecord(w.ev_fork, st));
            NL_TRY(join_ok(join.wait(q - 1)));  // the rest of update q - 1 wrote the cross's tiles
            NL_TRY(tc_gemm16_update(rest, rest, wd, L21, ld, utp, nb, A22, ld, st, w.flag, false, true));
            if (side_now) {
                const int m2 = rest - kLaTile;
                NL_TRY(join_ok(join.wait(q - 2)));  // ev_join[q % 2] is free again
                NL_CUDA_OK(cudaStreamWaitEvent(w.side, w.ev_fork, 0));
                // (a panel's time of slack: a quarter of the SMs, the rest left to concurrent solves' panels)
                NL_TRY(tc_gemm16_update(m2, m2, wd, L21 + (int64_t)kLaTile * ld, ld, utp + (int64_t)kLaTile * nb, nb,
                                        A22 + (int64_t)kLaTile * ld + kLaTile, ld, w.side, w.flag, false, false,
                                        std::max(1, num_sms() / 4)));
                NL_CUDA_OK(cudaEventRecord(w.ev_join[q & 1], w.side));
                join.pending |= 1 << (q & 1);
                ++nl;
            }
        }
        return NL_OK;
    };
    for (int K = 0; K < N; K += nb) {
        const int wd = std::min(nb, N - K), M = N - K;
        const int rest = N - K - wd;
        const bool tc = (gemm == 2) && std::is_same<S, __half>::value && (wd % 64 == 0);
        const size_t trsm_smem = (size_t)wd * wd * sizeof(T) + (size_t)wd * kTrsmThreads * sizeof(T);
        if (fast) {
            const int wp = (int)round_up(wd, 32);
            if constexpr (kHalf) {
                const int R = (rest > 0 && w.stream >= 0) ? panel16_fit_rows(rest, w.stream) : 0;
                if (R > 0) {
                    if (!pub_cleared) {
                        NL_CUDA_OK(cudaMemsetAsync(w.pub, 0, (size_t)128 * 128 * 8, st));
                        pub_cleared = true;
                    }
                    // the streamed rows and columns, then (if any) the rest in one off-diagonal launch
                    __half* utp = tc ? ut_of(K) : nullptr;
                    NL_TRY(launch_panel16(A, ld, K, wd, K + wd + R, ipiv, w, utp, nb, st, (K / nb) & 1));
                    if (R < rest) {
                        NL_TRY(launch_offdiag16<__half>(A, ld, K, wd, N, utp, nb, w.flag, (const float*)w.stage, -1,
                                                        0, st, R));
                        ++nl;
                    }
                    NL_TRY(update(K, wd, tc, utp));
                    nl += 2;
                    continue;
                }
                prof_begin("k_diag_lu16", st);
                k_diag_lu16<__half><<<1, kD16Threads, kDiag16Smem, st>>>(A, ld, K, wd, ipiv, w.flag, (float*)w.stage);
                prof_end("k_diag_lu16", st);
            } else {
                prof_begin("k_diag_lu", st);
                k_diag_lu<T, S, RND><<<1, kDiagThreads, (size_t)wp * (wp + 1) * sizeof(T), st>>>(A, ld, K, wd, ipiv,
                                                                                            w.flag, w.stage);
                prof_end("k_diag_lu", st);
            }
            ++nl;
            if (rest > 0) {
                if constexpr (kHalf) {
                    NL_TRY(launch_offdiag16<__half>(A, ld, K, wd, N, tc ? ut_of(K) : nullptr, nb, w.flag,
                                                    (const float*)w.stage, -1, 0, st));
                } else {
                    const int nrb = (int)cdiv(rest, kOffThreads / kOffG);
                    const size_t sm = (size_t)wp * wp * sizeof(T) + (size_t)wp * (kOffThreads / kOffG) * sizeof(T);
                    prof_begin("k_offdiag", st);
                    k_offdiag<T, S, RND><<<2 * nrb, kOffThreads, sm, st>>>(A, ld, K, wd, N, nrb, nullptr, nb, w.flag,
                                                                          w.stage);
                    prof_end("k_offdiag", st);
                }
                NL_TRY(update(K, wd, tc, ut_of(K)));
                nl += 2;
            }
            NL_CUDA_OK(cudaGetLastError());
            continue;
        }
        k_panel_load<T, S><<<M, 128, 0, st>>>(A, ld, K, M, wd, P, ldp);
        ++nl;
        for (int k0 = 0; k0 < wd; k0 += NBL) {
            const int wl = std::min(NBL, wd - k0);
            nl_status s = launch_leaf<T, NBL, RND>(P, ldp, k0, M, wd, wl, ipiv + K + k0, K + k0, w.info, st);
            if (s != NL_OK) return s;
            ++nl;
            if (k0 + wl < wd && M > k0 + wl) {
                unsigned g = (unsigned)cdiv(M - k0 - wl, 64);
                k_panel_gemm<T, NBL><<<g, 256, 0, st>>>(P, ldp, k0, wl, M, wd);
                ++nl;
            }
        }
        k_panel_store<T, S><<<M, 128, 0, st>>>(A, ld, K, M, wd, P, ldp);
        ++nl;
        if (N - wd > 0) {
            k_laswp<S><<<(unsigned)cdiv(N - wd, 256), 256, 0, st>>>(A, ld, K, wd, N, ipiv);
            ++nl;
        }
        if (rest > 0) {
            k_trsm_u12<T, S, RND><<<(unsigned)cdiv(rest, kTrsmThreads), kTrsmThreads, trsm_smem, st>>>(
                A, ld, K, wd, N, tc ? w.ut : nullptr, nb, nullptr);
            nl_status s = trailing_update<T, S>(N, A, ld, K, wd, nb, tc, w.ut, nullptr, st);
            if (s != NL_OK) return s;
            nl += 2;
        }
        NL_CUDA_OK(cudaGetLastError());
    }
    NL_TRY(join_ok(join.all()));
    if (launches) *launches += nl;
    return NL_OK;
}

// ------------------------------------------------------ two-level LU --
// Outer block W (a multiple of 128 up to 512), inner panels of 128, for the
// binary16 fast path: the arithmetic of rounding period W, i.e. the oracle's
// binary16-storage / binary32-arithmetic elimination with nb = W.  Per outer
// block [K0, K0 + W):
//   * its row and column strips (rows K0.. x columns K0..K0+W-1, and rows
//     K0..K0+W-1 x the columns right of it) are copied to a single-precision
//     shadow P;
//   * each inner panel is factored on P by the streaming panel (or the two
//     launches) exactly as the one-level path factors A: multipliers and U
//     entries rounded to binary16 as they are formed, U12^T of the columns
//     right of the outer block written in binary16 for the update below;
//   * the inner panel's update is applied in single precision, unrounded, to
//     the rest of the two strips only: with the SIMT update one fused
//     multiply-add per term in increasing k (the oracle's sequence exactly);
//     with the tensor-core update on the tcgen05 kernel for binary32 C (the
//     operands are binary16 values, so the K products are exact and their
//     sum is applied with one binary32 rounding);
//   * the strips go back to A (their entries are now binary16 values), and
//     the rest of the matrix receives one update of depth W,
//     A22 <- fl16(A22 - L21 U12), on the tensor cores (K streamed through the
//     persistent kernel's operand ring) or SIMT.
// So the trailing matrix is read and written once per W columns instead of
// once per 128.
template <bool TO32>
__global__ void __launch_bounds__(256) k_strip_copy(__half* __restrict__ A, int64_t lda, float* __restrict__ P,
                                                    int64_t ldp, int r0, int c0, int ncols)
{
    const int i = r0 + blockIdx.y;
    const int j = c0 + (blockIdx.x * 256 + threadIdx.x) * 8;
    if (j >= c0 + ncols) return;
    __half* a = A + (int64_t)i * lda + j;
    float* q = P + (int64_t)i * ldp + j;
    const int n = min(8, c0 + ncols - j);
    if (n == 8 && ((((uintptr_t)a) & 15) == 0) && ((((uintptr_t)q) & 15) == 0)) {
        float v[8];
        if (TO32) {
            load8(a, v);
            store8(q, v);
        } else {
            load8(q, v);
            store8(a, v);
        }
    } else {
        for (int e = 0; e < n; ++e) {
            if (TO32) q[e] = __half2float(a[e]);
            else a[e] = __float2half_rn(q[e]);
        }
    }
}

template <bool TO32>
static nl_status copy_block(__half* A, int64_t lda, float* P, int64_t ldp, int r0, int c0, int nrows, int ncols,
                            cudaStream_t st)
{
    if (nrows <= 0 || ncols <= 0) return NL_OK;
    for (int y0 = 0; y0 < nrows; y0 += 65535) {
        const int ny = std::min(65535, nrows - y0);
        k_strip_copy<TO32><<<dim3((unsigned)cdiv(ncols, 256 * 8), (unsigned)ny), 256, 0, st>>>(A, lda, P, ldp, r0 + y0,
                                                                                              c0, ncols);
    }
    NL_CUDA_OK(cudaGetLastError());
    return NL_OK;
}

static nl_status lu16_factor_2lvl(int N, __half* A, int64_t ld, int* ipiv, int W, int gemm, const LuWork& w,
                                  cudaStream_t st, int* launches)
{
    float* P = w.p32;
    const int64_t ldp = w.ldp32;
    if (!P) {
        set_error("lu16: an outer block above 128 needs the single-precision shadow workspace");
        return NL_EINVAL;
    }
    int nl = 0;
    NL_CUDA_OK(cudaMemsetAsync(w.info, 0, 10 * sizeof(int), st));  // info, flag, ..., the panel's role ticket
    NL_CUDA_OK(cudaMemsetAsync(w.pub, 0, (size_t)128 * 128 * 8, st));
    static bool smem_set = false;
    if (!smem_set) {
        if (set_max_dynamic_smem((const void*)k_offdiag16<float>) != NL_OK ||
            set_max_dynamic_smem((const void*)k_offdiag16<float, 256>) != NL_OK ||
            set_max_dynamic_smem((const void*)k_diag_lu16<float>) != NL_OK)
            return NL_ECUDA;
        smem_set = true;
    }
    for (int K0 = 0; K0 < N; K0 += W) {
        const int Wd = std::min(W, N - K0), far = N - K0 - Wd, C1 = K0 + Wd;
        const bool tc = gemm == 2 && tc_gemm_supported() && (Wd % 64 == 0);
        NL_TRY(copy_block<true>(A, ld, P, ldp, K0, K0, N - K0, Wd, st));
        NL_TRY(copy_block<true>(A, ld, P, ldp, K0, C1, Wd, far, st));
        nl += 2;
        for (int p0 = 0; p0 < Wd; p0 += 128) {
            const int K = K0 + p0, wd = std::min(128, Wd - p0), rest = N - K - wd;
            __half* ut = (tc && far > 0) ? w.ut : nullptr;
            const int R = (rest > 0 && w.stream >= 0) ? panel16_fit_rows(rest, w.stream) : 0;
            if (R > 0) {
                NL_TRY(launch_panel16<float>(P, ldp, K, wd, K + wd + R, ipiv, w, ut, W, st, (K / 128) & 1, C1, p0));
                ++nl;
                if (R < rest) {
                    NL_TRY(launch_offdiag16<float>(P, ldp, K, wd, N, ut, W, w.flag, (const float*)w.stage, C1, p0, st, R));
                    ++nl;
                }
            } else {
                prof_begin("k_diag_lu16", st);
                k_diag_lu16<float><<<1, kD16Threads, kDiag16Smem, st>>>(P, ldp, K, wd, ipiv, w.flag, (float*)w.stage);
                prof_end("k_diag_lu16", st);
                ++nl;
                if (rest > 0) {
                    NL_TRY(launch_offdiag16<float>(P, ldp, K, wd, N, ut, W, w.flag, (const float*)w.stage, C1, p0, st));
                    ++nl;
                }
            }
            // this inner panel's update on the rest of the two strips, unrounded (single
            // precision): SIMT fused multiply-adds in order k (the oracle's arithmetic), or
            // with the tensor-core update the tcgen05 kernel for binary32 C
            const bool tci = gemm == 2 && tc_gemm_supported();
            const int right = C1 - K - wd;  // strip columns right of the inner panel
            if (rest > 0 && right > 0) {
                const float* L21 = P + (K + wd) * ldp + K;
                const float* U12 = P + K * ldp + K + wd;
                float* C22 = P + (K + wd) * ldp + K + wd;
                if (tci) NL_TRY(tc_update_f32(rest, right, wd, L21, ldp, U12, ldp, C22, ldp, st, w.flag));
                else NL_TRY((launch_gemm_simt<float, float>(rest, right, wd, L21, ldp, U12, ldp, C22, ldp, st, w.flag)));
                ++nl;
            }
            const int below = C1 - K - wd;  // rows of the outer block below the inner panel
            if (far > 0 && below > 0) {
                const float* L21 = P + (K + wd) * ldp + K;
                const float* U12 = P + K * ldp + C1;
                float* C22 = P + (K + wd) * ldp + C1;
                if (tci) NL_TRY(tc_update_f32(below, far, wd, L21, ldp, U12, ldp, C22, ldp, st, w.flag));
                else NL_TRY((launch_gemm_simt<float, float>(below, far, wd, L21, ldp, U12, ldp, C22, ldp, st, w.flag)));
                ++nl;
            }
        }
        NL_TRY(copy_block<false>(A, ld, P, ldp, K0, K0, N - K0, Wd, st));
        NL_TRY(copy_block<false>(A, ld, P, ldp, K0, C1, Wd, far, st));
        nl += 2;
        if (far > 0) {
            __half* L21 = A + (int64_t)C1 * ld + K0;
            __half* A22 = A + (int64_t)C1 * ld + C1;
            if (tc) NL_TRY(tc_gemm16_update(far, far, Wd, L21, ld, w.ut, W, A22, ld, st, w.flag));
            else NL_TRY((launch_gemm_simt<__half, float>(far, far, Wd, L21, ld, A + (int64_t)K0 * ld + C1, ld, A22,
                                                        ld, st, w.flag)));
            ++nl;
        }
        NL_CUDA_OK(cudaGetLastError());
    }
    if (launches) *launches += nl;
    return NL_OK;
}

// Outer block nb: a multiple of 16 up to 128 (one level), or 256, 384, 512
// (two levels, fast path only; the interchanging path factors with 128).
bool lu16_nb_valid(int nb) { return (nb >= 16 && nb <= 128 && nb % 16 == 0) || nb == 256 || nb == 384 || nb == 512; }

nl_status lu16_factor(int N, __half* A, int64_t ld, int* ipiv, int nb, int gemm, bool fast, const LuWork& w,
                      cudaStream_t st, int* launches)
{
    if (!lu16_nb_valid(nb)) {
        set_error("lu16: nb must be a multiple of 16 in [16, 128], or 256, 384 or 512");
        return NL_EINVAL;
    }
    if (gemm == 2 && !tc_gemm_supported()) gemm = 1;
    if (nb > 128) {
        if (fast) return lu16_factor_2lvl(N, A, ld, ipiv, nb, gemm, w, st, launches);
        nb = 128;  // the interchanging path (partial pivoting needs row swaps): one level
    }
    return lu_factor_impl<float, __half, 16, true>(N, A, ld, ipiv, nb, gemm, fast, w, st, launches);
}

nl_status lu64_factor(int N, double* A, int64_t ld, int* ipiv, int nb, bool fast, const LuWork& w, cudaStream_t st,
                      int* launches)
{
    if (nb < 16 || nb > 128 || nb % 16) {
        set_error("lu64: nb must be a multiple of 16 in [16, 128]");
        return NL_EINVAL;
    }
    return lu_factor_impl<double, double, 8, false>(N, A, ld, ipiv, nb, 1, fast, w, st, launches);
}

// The single-precision factorisation of the two-precision F32 Newton method
// (Section 1.3): binary32 storage and arithmetic, always the interchanging
// path (leaf panels with pivot search, row swaps, U12 solve, SIMT update).
nl_status lu32_factor(int N, float* A, int64_t ld, int* ipiv, int nb, const LuWork& w, cudaStream_t st, int* launches)
{
    if (nb < 16 || nb > 128 || nb % 16) {
        set_error("lu32: nb must be a multiple of 16 in [16, 128]");
        return NL_EINVAL;
    }
    return lu_factor_impl<float, float, 16, false>(N, A, ld, ipiv, nb, 1, false, w, st, launches);
}

// ------------------------------------------------ binary16 arithmetic LU --
// Partial-pivot LU with every operation rounded to binary16, the arithmetic
// of the paper's F16 column (Section 1.3): at step k the pivot is the first
// row of largest |a_ik| (i >= k), rows k and p are swapped whole,
// l_ik = fl16(a_ik / a_kk) and a_ij <- fl16(a_ij - fl16(l_ik a_kj)) for
// i, j > k, so every entry takes its updates in increasing k.  One
// cooperative launch, one CTA per SM: a warp updates one row at a time, the
// next column's pivot candidates are formed during the update, and each step
// ends at a bounded grid barrier (one more after a row swap).  The product of
// two binary16 numbers is exact in binary32; the difference and the quotient
// are formed in binary32 and rounded once more, to binary16, which is the
// correctly rounded result (24 >= 2 * 11 + 2).  Matrix reads bypass L1
// (other SMs write the rows between barriers).
constexpr int kHaThreads = 512;
constexpr int kHaWarps = kHaThreads / 32;
constexpr int kHaU = 8;  // row entries per lane per batch of loads

__device__ __forceinline__ float h16r(float v) { return __half2float(__float2half_rn(v)); }

// {|a| bits, ~i}: the largest packed value is the first row of largest |a|.
__device__ __forceinline__ unsigned long long ha_pack(float a, int i)
{
    return ((unsigned long long)__float_as_uint(fabsf(a)) << 32) | (unsigned long long)(~(unsigned)i);
}

__device__ __forceinline__ unsigned long long ha_block_max(unsigned long long v, unsigned long long* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    __syncthreads();  // red is reused across calls
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    v = 0;
#pragma unroll
    for (int q = 0; q < kHaWarps; ++q) v = red[q] > v ? red[q] : v;
    return v;
}

// Grid barrier over co-resident CTAs: bar[0] counts arrivals, bar[1] is the
// generation (both zero at launch).  Bounded: false after recording a timeout,
// or when another CTA recorded an error.
__device__ bool ha_grid_sync(unsigned* bar, unsigned& gen, unsigned* err)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        if (atomicAdd(&bar[0], 1u) == gridDim.x - 1) {
            atomicExch(&bar[0], 0u);
            __threadfence();
            atomicAdd(&bar[1], 1u);
        } else {
            long long spins = 0;
            while ((unsigned)ld_acquire_gpu((const int*)&bar[1]) == gen) {
                if (*(volatile unsigned*)err) {
                    ok = 0;
                    break;
                }
                if (++spins > kSpinLimit) {
                    atomicOr(err, (unsigned)ERR_TIMEOUT_OTHER);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        ++gen;
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

__global__ void __launch_bounds__(kHaThreads, 1) k_lu16_arith(__half* __restrict__ A, int64_t lda, int N,
                                                              int* __restrict__ ipiv, int* __restrict__ info,
                                                              unsigned* __restrict__ bar,
                                                              unsigned long long* __restrict__ cand,
                                                              unsigned* __restrict__ err)
{
    __shared__ unsigned long long red[kHaWarps];
    const int tid = threadIdx.x, lane = tid & 31;
    const int G = gridDim.x;
    const int gw = blockIdx.x * kHaWarps + (tid >> 5), nw = G * kHaWarps;  // this warp, all warps
    unsigned gen = 0;
    // pivot candidates of column 0
    unsigned long long nb = 0;
    if (lane == 0)
        for (int i = gw; i < N; i += nw) {
            const unsigned long long c = ha_pack(__half2float(__ldcg(A + (int64_t)i * lda)), i);
            nb = c > nb ? c : nb;
        }
    nb = ha_block_max(nb, red);
    if (tid == 0) cand[blockIdx.x] = nb;
    if (!ha_grid_sync(bar, gen, err)) return;
    for (int k = 0; k < N; ++k) {
        unsigned long long b = 0;
        for (int g = tid; g < G; g += kHaThreads) {
            const unsigned long long c = __ldcg(cand + (k & 1) * G + g);
            b = c > b ? c : b;
        }
        b = ha_block_max(b, red);
        const int p = (int)(~(unsigned)(b & 0xffffffffull));
        if (blockIdx.x == 0 && tid == 0) ipiv[k] = p;
        if (p != k && p > k && p < N) {  // swap rows k and p whole
            __half* Rk = A + (int64_t)k * lda;
            __half* Rp = A + (int64_t)p * lda;
            for (int j = blockIdx.x * kHaThreads + tid; j < N; j += G * kHaThreads) {
                const __half t = __ldcg(Rk + j);
                Rk[j] = __ldcg(Rp + j);
                Rp[j] = t;
            }
            if (!ha_grid_sync(bar, gen, err)) return;
        }
        const __half* Rk = A + (int64_t)k * lda;
        const float akk = __half2float(__ldcg(Rk + k));
        if (akk == 0.0f && blockIdx.x == 0 && tid == 0) atomicCAS(info, 0, k + 1);
        if (k == N - 1) break;
        nb = 0;
        if (akk == 0.0f) {  // no elimination at this step; the next column's candidates as they stand
            if (lane == 0)
                for (int i = k + 1 + gw; i < N; i += nw) {
                    const unsigned long long c = ha_pack(__half2float(__ldcg(A + (int64_t)i * lda + k + 1)), i);
                    nb = c > nb ? c : nb;
                }
        } else {
            bool inf = false;
            for (int i = k + 1 + gw; i < N; i += nw) {
                __half* Ri = A + (int64_t)i * lda;
                const float l = h16r(__fdiv_rn(__half2float(__ldcg(Ri + k)), akk));
                __syncwarp();  // every lane has read a_ik before lane 0 overwrites it
                if (lane == 0) Ri[k] = __float2half_rn(l);
                // kHaU entries per lane: all loads issued before the stores (the rows may alias
                // as far as the compiler knows), the same operations per entry
                for (int j0 = k + 1; j0 < N; j0 += 32 * kHaU) {
                    __half rk[kHaU], ri[kHaU];
#pragma unroll
                    for (int u = 0; u < kHaU; ++u) {
                        const int j = j0 + u * 32 + lane;
                        rk[u] = j < N ? __ldcg(Rk + j) : __ushort_as_half((unsigned short)0);
                        ri[u] = j < N ? __ldcg(Ri + j) : __ushort_as_half((unsigned short)0);
                    }
#pragma unroll
                    for (int u = 0; u < kHaU; ++u) {
                        const int j = j0 + u * 32 + lane;
                        if (j < N) {
                            const float pr = h16r(l * __half2float(rk[u]));
                            const float v = h16r(__half2float(ri[u]) - pr);
                            Ri[j] = __float2half_rn(v);
                            inf |= isinf(v);
                            if (j == k + 1) {
                                const unsigned long long c = ha_pack(v, i);
                                nb = c > nb ? c : nb;
                            }
                        }
                    }
                }
            }
            if (inf) atomicOr(info + 1, 1);
        }
        nb = ha_block_max(nb, red);
        if (tid == 0) cand[((k + 1) & 1) * G + blockIdx.x] = nb;
        if (!ha_grid_sync(bar, gen, err)) return;
    }
}

nl_status lu16_factor_arith(int N, __half* A, int64_t ld, int* ipiv, const LuWork& w, cudaStream_t st)
{
    static std::atomic<int> grid_cache{0};
    int grid = grid_cache.load();
    if (grid == 0) {
        int per_sm = 0;
        NL_CUDA_OK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lu16_arith, kHaThreads, 0));
        if (per_sm < 1) {
            set_error("binary16-arithmetic LU: the kernel does not fit on an SM");
            return NL_ECUDA;
        }
        grid = std::min(num_sms(), 128 * 128 / 2);  // one CTA per SM; two candidate rows per CTA fit in pub
        grid_cache.store(grid);
    }
    NL_CUDA_OK(cudaMemsetAsync(w.info, 0, 6 * sizeof(int), st));  // info, overflow, (err), barrier count and generation
    unsigned* err = tc_error_word();
    if (!err) err = (unsigned*)(w.info + 2);
    unsigned* bar = (unsigned*)(w.info + 4);
    int* info = w.info;
    unsigned long long* cand = w.pub;
    int Nv = N;
    int64_t ldv = ld;
    void* args[] = {(void*)&A, (void*)&ldv, (void*)&Nv, (void*)&ipiv, (void*)&info, (void*)&bar, (void*)&cand,
                    (void*)&err};
    NL_CUDA_OK(cudaLaunchCooperativeKernel((const void*)k_lu16_arith, dim3(grid), dim3(kHaThreads), args, 0, st));
    return NL_OK;
}

}  // namespace nl

// ================================================================ grouped ==
// Many independent matrices of different N factored in lock step: outer step
// k launches the diagonal-block kernel for every matrix with N > k nb, the
// off-diagonal solves of all of them, and their trailing updates, each as one
// launch over a precomputed task list (largest matrices first).  The kernels
// are the single-matrix fast-path bodies; a matrix whose flag word is non-zero
// (fast path failed, or marked to be skipped) does no work.  No interchanges:
// a matrix that needs them is left with bit 0 of its flag set.
namespace nl {

size_t lu_stage_bytes() { return (size_t)2 * 128 * 128 * 8 + 128 * 8; }

template <typename T, typename S, bool RND>
__global__ void __launch_bounds__(kDiagThreads, 1) k_diag_lu_g(const GInst* __restrict__ inst,
                                                               const GTask* __restrict__ tasks, int K, int nb)
{
    const GInst I = inst[tasks[blockIdx.x].inst];
    diag_lu_body<T, S, RND>(reinterpret_cast<S*>(I.A), I.ld, K, min(nb, I.N - K), I.ipiv, I.flag, I.stage);
}

__global__ void __launch_bounds__(kD16Threads, 1) k_diag_lu16_g(const GInst* __restrict__ inst,
                                                                const GTask* __restrict__ tasks, int K, int nb)
{
    const GInst I = inst[tasks[blockIdx.x].inst];
    diag_lu16_body(reinterpret_cast<__half*>(I.A), I.ld, K, min(nb, I.N - K), I.ipiv, I.flag,
                   reinterpret_cast<float*>(I.stage));
}

template <typename T, typename S, bool RND>
__global__ void __launch_bounds__(kOffThreads) k_offdiag_g(const GInst* __restrict__ inst,
                                                           const GTask* __restrict__ tasks, int K, int nb)
{
    const GTask t = tasks[blockIdx.x];
    const GInst I = inst[t.inst];
    offdiag_body<T, S, RND>(reinterpret_cast<S*>(I.A), I.ld, K, nb, I.N, t.b, nullptr, nb, I.flag, I.stage, t.a);
}

__global__ void __launch_bounds__(kO16Threads) k_offdiag16_g(const GInst* __restrict__ inst,
                                                             const GTask* __restrict__ tasks, int K, int nb, int tc)
{
    const GTask t = tasks[blockIdx.x];
    const GInst I = inst[t.inst];
    offdiag16_body(reinterpret_cast<__half*>(I.A), I.ld, K, nb, I.N, t.b, tc ? I.ut : nullptr, nb, I.flag,
                   reinterpret_cast<const float*>(I.stage), t.a);
}

template <typename S, typename T>
__global__ void __launch_bounds__(256) k_gemm_simt_g(const GInst* __restrict__ inst, const GTask* __restrict__ tasks,
                                                     int K, int w)
{
    const GTask t = tasks[blockIdx.x];
    const GInst I = inst[t.inst];
    const int rest = I.N - K - w;
    S* A = reinterpret_cast<S*>(I.A);
    const int64_t ld = I.ld;
    gemm_simt_body<S, T>(rest, rest, w, A + (int64_t)(K + w) * ld + K, ld, A + (int64_t)K * ld + K + w, ld,
                         A + (int64_t)(K + w) * ld + K + w, ld, I.flag, t.a, t.b);
}

// ------------------------------------------- persistent grouped LU --
// The whole grouped factorisation in one launch: CTAs (one per SM) take tasks
// from a device queue in order (an atomic counter) and each task waits, with
// a bounded poll, for the progress word of its matrix:
//   diag(i, k)      needs phase 3k   (matrix i's update of step k-1 done),
//   offdiag(i, k)   needs phase 3k+1 (its diagonal block factored),
//   update(i, k)    needs phase 3k+2 (all its off-diagonal solves done);
// the last task of each phase advances the word (release).  The queue lists
// step k's diagonal tasks, then its off-diagonal tasks, then its update
// tiles, step by step, so every task's dependencies come earlier in the queue
// and were taken by CTAs that are running: no co-residency is needed and the
// launch can be captured in a graph.  A CTA of 512 threads runs a diagonal
// block (diag_lu16_body), four off-diagonal blocks of one role side by side
// (four groups of 128 threads, each with its own shared region; padding
// groups get blocks past the matrix and store nothing), or one update tile of
// TM x 64 with sequential single-precision fused multiply-adds over k and one
// rounding to binary16: the arithmetic of the three-launch SIMT path, so the
// factors are bitwise those of the single-matrix LU with the SIMT update.
// A matrix whose fast path failed (flag set) skips its work but its tasks
// still advance its progress word; a wait that gives up records the error
// and its CTA skips the work the same way, so nothing waits forever.
constexpr int kPgThreads = 512;
constexpr long long kPgSpin = 1LL << 24;

// A queue entry carries its matrix's pointers (one 80-byte record, fetched
// ahead with cp.async while the previous task runs).
struct alignas(16) PTask {
    void* A;
    int* ipiv;
    int* flag;
    void* stage;
    __half* ut;
    int ld, N;
    int inst, kind, step, a, b, n;  // kind 0 diag; 1 off-diagonal quad (a first block, b blocks in it,
                                    // n = 1 row role / 0 column role); 2 update tile (a = m0, b = n0)
};
static_assert(sizeof(PTask) == 80, "queue entries are five 16-byte chunks");

// progress word: the phase reached, with kPgFail once the matrix's flag is set
// (folded in by the task that completes each phase, so a waiting task learns
// both from its one acquire load)
constexpr int kPgFail = 1 << 30;

// Polls before a wait gives up: 0 = kPgSpin; negative = give up at the first
// unmet poll (a test of the timeout path that needs no fault: a wait that runs
// out whatever the producers do).
__device__ long long g_pg_spin_limit = 0;

__device__ __forceinline__ bool pg_wait(const int* p, int need, unsigned* err, int* val)
{
    long long it = 0;
    int v;
    const long long lim = g_pg_spin_limit;
    const long long limit = lim == 0 ? kPgSpin : (lim < 0 ? 0 : lim);
    while (((v = ld_acquire_gpu(p)) & ~kPgFail) < need) {
        if (*(volatile unsigned*)err) return false;
        if (++it > limit) {
            atomicOr(err, (unsigned)ERR_TIMEOUT_OTHER);
            return false;
        }
        __nanosleep(64);
    }
    *val = v;
    return true;
}

__device__ __forceinline__ int atom_add_acq_rel_gpu(int* p, int v)
{
    int old;
    asm volatile("atom.add.acq_rel.gpu.global.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// thread 0: queue entry t (if any) into a shared slot, asynchronously
__device__ __forceinline__ void pg_fetch(const PTask* tasks, int t, int ntasks, PTask* slot)
{
    if (t < ntasks) {
        const char* src = reinterpret_cast<const char*>(tasks + t);
        const uint32_t dst = smem_u32(slot);
#pragma unroll
        for (int q = 0; q < 5; ++q)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + 16 * q), "l"(src + 16 * q) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// C[m0.., n0..] (TM x 64) <- fl16(C - A B) over K, 512 threads: thread (ty, tx) =
// (tid / 16, tid % 16) owns rows ty + 32 a and columns tx + 16 b; every entry takes
// its K products in increasing k, one fused multiply-add each.  The operands are
// written by other CTAs of the same launch, so they are read through plain
// (coherent) loads, never the read-only path.
template <int TM>
__device__ __forceinline__ void pg_gemm_tile(int M, int Nc, int K, const __half* A, int64_t lda, const __half* B,
                                             int64_t ldb, __half* C, int64_t ldc, int m0, int n0, float* sm)
{
    constexpr int BK = 16, RA = TM / 32;
    float* As = sm;                    // [BK][TM + 1]
    float* Bs = sm + BK * (TM + 1);    // [BK][64]
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    float acc[RA][4];
#pragma unroll
    for (int a = 0; a < RA; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = m0 + ty + 32 * a, j = n0 + tx + 16 * b;
            acc[a][b] = (i < M && j < Nc) ? __half2float(C[(int64_t)i * ldc + j]) : 0.0f;
        }
    for (int k0 = 0; k0 < K; k0 += BK) {
        __syncthreads();
        for (int q = tid; q < TM * BK; q += kPgThreads) {
            const int r = q / BK, kk = q % BK, i = m0 + r, k = k0 + kk;
            As[kk * (TM + 1) + r] = (i < M && k < K) ? __half2float(A[(int64_t)i * lda + k]) : 0.0f;
        }
        for (int q = tid; q < BK * 64; q += kPgThreads) {
            const int kk = q / 64, x = q % 64, k = k0 + kk, j = n0 + x;
            Bs[kk * 64 + x] = (k < K && j < Nc) ? __half2float(B[(int64_t)k * ldb + j]) : 0.0f;
        }
        __syncthreads();
        const int kmax = min(BK, K - k0);
        for (int kk = 0; kk < kmax; ++kk) {
            float av[RA], bv[4];
#pragma unroll
            for (int a = 0; a < RA; ++a) av[a] = As[kk * (TM + 1) + ty + 32 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[kk * 64 + tx + 16 * b];
#pragma unroll
            for (int a = 0; a < RA; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(-av[a], bv[b], acc[a][b]);
        }
    }
#pragma unroll
    for (int a = 0; a < RA; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = m0 + ty + 32 * a, j = n0 + tx + 16 * b;
            if (i < M && j < Nc) C[(int64_t)i * ldc + j] = __float2half_rn(acc[a][b]);
        }
}

constexpr long long kPgTcWait = 2000000000LL;  // cycles: bounded mbarrier waits of the tcgen05 tiles

// One 128 x 128 update tile on the tensor cores (TC kernels): thread 0 loads the
// 64-wide A slab (L21 rows, through the matrix's tensor map) and B slab (U12^T
// rows, through its U12^T map) with TMA, issues the four K = 16 tcgen05.mma of
// the slab into the CTA's 128-column TMEM accumulator and commits them; each of
// the 16 warps then reads its 32 lanes x 32 columns (warp w: lanes 32 (w % 4),
// columns 32 (w / 4)) and writes C = fl16(C - acc).  The per-element arithmetic
// is the trailing-update kernels' (same MMAs in the same order, one
// subtraction, one rounding).  `uses` counts the tiles issued by this CTA (the
// mbarrier phases); a wait that gives up marks the CTA dead: its later tiles
// store nothing and it never touches its barriers again.
__device__ __forceinline__ void pg_tc_tile(__half* A, int64_t ld, const TmapBytes* __restrict__ maps, int inst, int K, int w,
                                           int rest, int m0, int n0, bool run, uint32_t tmem, uint32_t& uses,
                                           uint64_t* tbar, int* dead, float* pgsm, unsigned* err)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t raw = smem_u32(pgsm), base = (raw + 1023u) & ~1023u;
    const uint32_t sA = base, sB = base + 128 * 128;
    const uint32_t bl = smem_u32(&tbar[0]), bm = smem_u32(&tbar[1]);
    const uint32_t ph = uses & 1u;
    // this CTA's earlier generic writes to the shared region, before the TMA writes into it
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    run = run && !*(volatile int*)dead;  // CTA-uniform: written by thread 0 only, read after a barrier
    if (run && threadIdx.x == 0) {
        const CUtensorMap* ma = reinterpret_cast<const CUtensorMap*>(&maps[2 * inst]);
        const CUtensorMap* mb = reinterpret_cast<const CUtensorMap*>(&maps[2 * inst + 1]);
        asm volatile("fence.proxy.async.global;" ::: "memory");  // the acquired operands, for the async proxy
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bl), "r"(2u * 128 * 128)
                     : "memory");
        tma_load_2d(sA, ma, K, K + w + m0, bl);
        tma_load_2d(sB, mb, 0, n0, bl);
        if (!mbar_wait(bl, ph, kPgTcWait)) {
            atomicOr(err, (unsigned)ERR_TIMEOUT_OTHER);
            *(volatile int*)dead = 1;
            mbar_wait(bl, ph, kPgTcWait);  // let copies in flight land
        } else {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            constexpr uint32_t idesc = tc_idesc_mn(128, 128);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint64_t ad = sw128_desc(sA + kk * 32), bd = sw128_desc(sB + kk * 32);
                const uint32_t acc = kk ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bm)
                         : "memory");
        }
    }
    // the epilogue's C segment does not depend on the MMAs: load it while they run
    const int q = warp & 3, cg = warp >> 2;
    const int row = m0 + q * 32 + lane, col0 = n0 + cg * 32;
    __half* Crow = A + (int64_t)(K + w + min(row, rest - 1)) * ld + K + w;
    const bool full = run && row < rest && col0 + 32 <= rest;
    uint4 cpre[4];
    if (full) {
        const uint4* p = reinterpret_cast<const uint4*>(Crow + col0);
#pragma unroll
        for (int v = 0; v < 4; ++v) cpre[v] = p[v];
    }
    __syncthreads();
    bool good = run && !*(volatile int*)dead;  // CTA-uniform (a failed load wait set it)
    const bool waited = good ? mbar_wait(bm, ph, kPgTcWait) : true;
    if (__syncthreads_or(!waited)) {
        if (threadIdx.x == 0) {
            atomicOr(err, (unsigned)ERR_TIMEOUT_OTHER);
            *(volatile int*)dead = 1;
            mbar_wait(bm, ph, kPgTcWait);  // let the MMAs in flight finish
        }
        good = false;
    }
    if (run) uses += 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (good) {
        uint32_t r[32];
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(cg * 32);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
              "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
              "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (full) {
            uint4* p = reinterpret_cast<uint4*>(Crow + col0);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                uint32_t wds[4] = {cpre[v].x, cpre[v].y, cpre[v].z, cpre[v].w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    __half2 h2;
                    memcpy(&h2, &wds[e], 4);
                    float2 f = __half22float2(h2);
                    f.x -= __uint_as_float(r[v * 8 + 2 * e]);
                    f.y -= __uint_as_float(r[v * 8 + 2 * e + 1]);
                    h2 = __floats2half2_rn(f.x, f.y);
                    memcpy(&wds[e], &h2, 4);
                }
                p[v] = make_uint4(wds[0], wds[1], wds[2], wds[3]);
            }
        } else if (run && row < rest) {
#pragma unroll
            for (int e = 0; e < 32; ++e)
                if (col0 + e < rest)
                    Crow[col0 + e] = __float2half_rn(__half2float(Crow[col0 + e]) - __uint_as_float(r[e]));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// ctl: [0] the queue's next task, [1 .. count] progress words, [1 + count .. 1 + 2 count)
// per-matrix task counters (set by k_pg_init before each launch).  TC: update tiles of
// 128 x 128 on the tensor cores (nb = 64, U12^T written by the column-role solves,
// tensor maps in `maps`); otherwise tm x 64 SIMT tiles.  Thread 0 takes the next queue
// index while it waits for the current task's dependencies and fetches that entry with
// cp.async while the task runs; a phase is handed on with an acquire-release count and
// a release store of the progress word.
template <bool TC>
__global__ void __launch_bounds__(kPgThreads, 1) k_lu_grouped_p(const PTask* __restrict__ tasks, int ntasks, int nb,
                                                                int tm, int tn, const TmapBytes* __restrict__ maps,
                                                                int* __restrict__ ctl, int count,
                                                                unsigned* __restrict__ err,
                                                                unsigned long long* __restrict__ tstat)
{
    extern __shared__ __align__(16) float pgsm[];
    __shared__ PTask qbuf[2];
    __shared__ int qidx[2], go, dead;
    __shared__ __align__(8) uint64_t tbar[2];  // TC: operands landed, MMAs done
    __shared__ uint32_t tslot;
    int* next = ctl;
    int* prog = ctl + 1;
    int* cnt = ctl + 1 + count;
    uint32_t tmem = 0, uses = 0;
    if constexpr (TC) {
        if ((threadIdx.x >> 5) == 0) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                         "r"(128u));
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
        }
        if (threadIdx.x == 32) {
            dead = 0;
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tbar[0])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tbar[1])));
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        tmem = tslot;
    }
    if (threadIdx.x == 0) {
        const int t0 = atomicAdd(next, 1);
        qidx[0] = t0;
        pg_fetch(tasks, t0, ntasks, &qbuf[0]);
        asm volatile("cp.async.wait_all;" ::: "memory");
    }
    int slot = 0;
    for (;;) {
        __syncthreads();
        const int t = qidx[slot];
        if (t >= ntasks) break;
        const PTask& T = qbuf[slot];  // stays put while the task runs (the prefetch fills the other slot)
        const int K = T.step * nb, w = min(nb, T.N - K), rest = T.N - K - w;
        __half* A = reinterpret_cast<__half*>(T.A);
        long long c0 = 0, c1 = 0;  // task timing (tstat): start, dependencies met
        if (threadIdx.x == 0) {
            c0 = clock64();
            const int tnext = atomicAdd(next, 1);  // its latency overlaps the wait below
            int v = 0;
            const bool ok = pg_wait(&prog[T.inst], 3 * T.step + T.kind, err, &v);
            c1 = clock64();
            go = (ok && !(v & kPgFail)) ? 1 : 0;
            qidx[slot ^ 1] = tnext;
            pg_fetch(tasks, tnext, ntasks, &qbuf[slot ^ 1]);  // lands while this task runs
        }
        __syncthreads();
        int* done_word = nullptr;  // thread 0: the counter this task adds to, and by how much
        int add = 0, total = 0, phase = 0;
        if (T.kind == 0) {
            if (go) diag_lu16_body<false, __half>(A, T.ld, K, w, T.ipiv, T.flag, reinterpret_cast<float*>(T.stage));
            phase = rest > 0 ? 3 * T.step + 1 : 3 * T.step + 3;
        } else if (T.kind == 1) {
            const int wp = (w + 31) & ~31;
            const int q = threadIdx.x >> 7, b = T.a + q;
            const int fl = (int)(offdiag16_smem(wp) / sizeof(float));
            if (go)
                offdiag16_body<__half>(A, T.ld, K, w, T.N, T.n ? (1 << 20) : 0, TC ? T.ut : nullptr, nb, T.flag,
                                       reinterpret_cast<const float*>(T.stage), b, -1, 0, threadIdx.x & 127,
                                       pgsm + q * fl);
            done_word = &cnt[T.inst];
            add = T.b;
            total = 2 * ((rest + kO16Rows - 1) / kO16Rows);
            phase = 3 * T.step + 2;
        } else {
            if constexpr (TC) {
                pg_tc_tile(A, T.ld, maps, T.inst, K, w, rest, T.a, T.b, go != 0, tmem, uses, tbar, &dead, pgsm, err);
            } else if (go) {
                const __half* L21 = A + (int64_t)(K + w) * T.ld + K;
                const __half* U12 = A + (int64_t)K * T.ld + K + w;
                __half* C = A + (int64_t)(K + w) * T.ld + K + w;
                if (tm == 128) pg_gemm_tile<128>(rest, rest, w, L21, T.ld, U12, T.ld, C, T.ld, T.a, T.b, pgsm);
                else pg_gemm_tile<64>(rest, rest, w, L21, T.ld, U12, T.ld, C, T.ld, T.a, T.b, pgsm);
            }
            done_word = &cnt[T.inst];
            add = 1;
            total = ((rest + tm - 1) / tm) * ((rest + tn - 1) / tn);
            phase = 3 * T.step + 3;
        }
        // TC: the off-diagonal solves' generic writes (L21 rows and U12^T, the tiles' TMA
        // operands) ordered before the TMA reads of them; the diagonal blocks and the
        // tiles' C are read by generic loads only
        if constexpr (TC)
            if (T.kind == 1) asm volatile("fence.proxy.async.global;" ::: "memory");
        if (threadIdx.x == 0) asm volatile("cp.async.wait_all;" ::: "memory");  // the next entry has landed
        __syncthreads();
        if (threadIdx.x == 0) {
            // the CTA's writes are ordered before thread 0's release by the barrier
            bool last = true;
            if (done_word) {
                last = atom_add_acq_rel_gpu(done_word, add) + add == total;
                if (last) *done_word = 0;
            }
            if (last) st_release_gpu(&prog[T.inst], phase | (*(volatile const int*)T.flag ? kPgFail : 0));
            if (tstat) {  // per kind: tasks, cycles waiting for dependencies, cycles working
                const long long c2 = clock64();
                atomicAdd(&tstat[3 * T.kind], 1ull);
                atomicAdd(&tstat[3 * T.kind + 1], (unsigned long long)(c1 - c0));
                atomicAdd(&tstat[3 * T.kind + 2], (unsigned long long)(c2 - c1));
            }
        }
        slot ^= 1;
    }
    if constexpr (TC) {
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if ((threadIdx.x >> 5) == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128u));
        }
    }
}

// Per-task timing of the persistent launch (off unless switched on): per task
// kind, the tasks run, the cycles spent waiting for their dependencies and the
// cycles spent on them (thread 0's clock64 from dependencies met to hand-off).
__device__ unsigned long long g_pg_tstat[9];
static std::atomic<bool> g_pg_tstat_on{false};

static unsigned long long* pg_task_stats_ptr()
{
    if (!g_pg_tstat_on.load()) return nullptr;
    void* p = nullptr;
    return cudaGetSymbolAddress(&p, g_pg_tstat) == cudaSuccess ? static_cast<unsigned long long*>(p) : nullptr;
}

// Before each launch: the queue counter and task counters zeroed, each progress
// word 0 with kPgFail for a matrix whose flag is already set (skipped).
__global__ void k_pg_init(int* __restrict__ ctl, int count, const GInst* __restrict__ inst)
{
    for (int i = threadIdx.x; i < 1 + 2 * count; i += blockDim.x) {
        int v = 0;
        if (i >= 1 && i <= count && *(volatile const int*)inst[i - 1].flag) v = kPgFail;
        ctl[i] = v;
    }
}

static size_t pg_smem_bytes(int nb)
{
    const int wp = (int)round_up(nb, 32);
    size_t b = std::max<size_t>(kDiag16Smem, 4 * offdiag16_smem(wp));
    b = std::max<size_t>(b, (size_t)(16 * (128 + 1) + 16 * 64) * sizeof(float));
    b = std::max<size_t>(b, 1024 + 2 * 128 * 128);  // the tcgen05 tile's A and B slabs, 1024-byte aligned
    return b;
}

// The persistent launch's queue order: a list schedule simulated on the host
// with a cost model (microseconds per task on one CTA).  `workers` CTAs; the
// tasks of a matrix's next phase become ready when its current phase is done
// (diagonal block -> off-diagonal quads -> update tiles -> next diagonal
// block); a free CTA takes the ready task whose matrix has the most outer
// steps left (the longest remaining chain), a diagonal block before quads
// before tiles, then in generation order.  The queue lists the tasks by
// simulated start, so every task's dependencies come earlier in it, and the
// long chains of the largest matrices advance while the others fill the gaps.
static std::vector<PTask> lu_grouped_schedule(int count, const GInst* host_inst, int nb, int tm, int tn, bool tc,
                                              int workers)
{
    struct Ready {
        int rem, kind;
        long long seq;
        PTask t;
        bool operator<(const Ready& o) const  // max-heap: most steps left, then kind, then earliest
        {
            if (rem != o.rem) return rem < o.rem;
            if (kind != o.kind) return kind > o.kind;
            return seq > o.seq;
        }
    };
    struct Busy {
        double end;
        int inst;
        bool operator<(const Busy& o) const { return end > o.end; }  // min-heap on finish time
    };
    std::vector<int> steps(count), step(count, 0), left(count, 0);
    std::priority_queue<Ready> ready;
    std::priority_queue<Busy> busy;
    long long seq = 0;
    size_t total = 0;
    for (int i = 0; i < count; ++i) steps[i] = (int)cdiv(host_inst[i].N, nb);
    // per-task times measured on a GB300 for w = 64 (clock64 around each task of the
    // 512-instance workload): diagonal block ~30 us, off-diagonal quad ~25 us, tile
    // ~6 us (tcgen05 128 x 128), ~15 us (SIMT 128 x 64), ~8 us (SIMT 64 x 64)
    auto dur = [&](int kind, int w) {
        const double f = (double)w / 64.0;
        if (kind == 0) return 0.47 * w;
        if (kind == 1) return 3.0 + 22.0 * f * f;
        return tc ? 6.0 : (tm == 128 ? 15.0 : 8.0) * f;
    };
    std::vector<double> tdur;  // per generated task, indexed by its seq
    auto mk = [&](int i, int kind, int k, int a, int b, int n) {
        const GInst& G = host_inst[i];
        PTask t;
        t.A = G.A;
        t.ipiv = G.ipiv;
        t.flag = G.flag;
        t.stage = G.stage;
        t.ut = G.ut;
        t.ld = (int)G.ld;
        t.N = G.N;
        t.inst = i;
        t.kind = kind;
        t.step = k;
        t.a = a;
        t.b = b;
        t.n = n;
        return t;
    };
    // phase `kind` of matrix i's current step becomes ready
    auto release = [&](int i, int kind) {
        const int k = step[i], K = k * nb, w = std::min(nb, host_inst[i].N - K), rest = host_inst[i].N - K - w;
        const int rem = steps[i] - k;
        auto push = [&](PTask t) {
            ready.push({rem, kind, seq++, t});
            tdur.push_back(dur(kind, w));
            left[i] += 1;
            total += 1;
        };
        if (kind == 0) {
            push(mk(i, 0, k, 0, 0, 0));
        } else if (kind == 1) {
            const int nblk = (int)cdiv(rest, kO16Rows);
            for (int role = 1; role >= 0; --role)
                for (int a = 0; a < nblk; a += 4) push(mk(i, 1, k, a, std::min(4, nblk - a), role));
        } else {
            for (int m0 = 0; m0 < rest; m0 += tm)
                for (int n0 = 0; n0 < rest; n0 += tn) push(mk(i, 2, k, m0, n0, 0));
        }
    };
    for (int i = 0; i < count; ++i) release(i, 0);
    std::vector<PTask> q;
    double t = 0.0;
    int idle = std::max(1, workers);
    while (!ready.empty() || !busy.empty()) {
        while (idle > 0 && !ready.empty()) {
            const Ready r = ready.top();
            ready.pop();
            q.push_back(r.t);
            busy.push({t + tdur[(size_t)r.seq], r.t.inst + count * r.t.kind});
            idle -= 1;
        }
        if (busy.empty()) break;
        const Busy b = busy.top();
        busy.pop();
        t = b.end;
        idle += 1;
        const int i = b.inst % count, kind = b.inst / count;
        if (--left[i] > 0) continue;
        // matrix i's phase `kind` is done
        const int K = step[i] * nb, rest = host_inst[i].N - K - std::min(nb, host_inst[i].N - K);
        if (kind == 0) {
            if (rest > 0) release(i, 1);
        } else if (kind == 1) {
            release(i, 2);
        } else {
            step[i] += 1;
            release(i, 0);
        }
    }
    return q;
}

// The persistent launch's queue (see lu_grouped_schedule).
static nl_status lu_grouped_plan_p(int count, const GInst* host_inst, int nb, int gemm, int tm, GroupPlan* plan)
{
    const int tn = gemm == 2 ? 128 : 64;
    if (gemm == 2) tm = 128;
    int nmax = 0;
    for (int i = 0; i < count; ++i) nmax = std::max(nmax, host_inst[i].N);
    const int steps = (int)cdiv(nmax, nb);
    const int workers = num_sms();
    std::vector<PTask> q = lu_grouped_schedule(count, host_inst, nb, tm, tn, gemm == 2, workers);
    lu_grouped_free(plan);
    plan->count = count;
    plan->nb = nb;
    plan->gemm = gemm;
    plan->steps = steps;
    plan->fp64 = false;
    plan->kind = 1;
    plan->tm = tm;
    plan->tn = tn;
    plan->off.clear();
    plan->n.clear();
    plan->nptasks = (int)q.size();
    plan->grid = std::max(1, std::min(plan->nptasks, num_sms()));
    std::vector<TmapBytes> maps;
    if (gemm == 2) {
        maps.resize(2 * (size_t)count);
        for (int i = 0; i < count; ++i)
            if (host_inst[i].N > nb && !tc_encode_instance_maps(reinterpret_cast<const __half*>(host_inst[i].A),
                                                                host_inst[i].N, host_inst[i].ld, host_inst[i].ut, nb,
                                                                &maps[2 * (size_t)i])) {
                set_error("grouped LU: tensor-map encoding failed for matrix %d", i);
                return NL_ECUDA;
            }
    }
    const size_t qb = q.size() * sizeof(PTask), cb = (size_t)(1 + 2 * count) * sizeof(int);
    const size_t mb = maps.size() * sizeof(TmapBytes);
    plan->bytes = round_up(qb, 256) + round_up(cb, 256) + mb;
    void* p = nullptr;
    NL_CUDA_OK(cudaMalloc(&p, plan->bytes));
    plan->tasks = reinterpret_cast<GTask*>(p);  // the allocation's base (freed through it)
    plan->ptasks = reinterpret_cast<PTask*>(p);
    plan->ctl = reinterpret_cast<int*>((char*)p + round_up(qb, 256));
    plan->maps = mb ? reinterpret_cast<TmapBytes*>((char*)p + round_up(qb, 256) + round_up(cb, 256)) : nullptr;
    if (qb) NL_CUDA_OK(cudaMemcpy(plan->ptasks, q.data(), qb, cudaMemcpyHostToDevice));
    if (mb) NL_CUDA_OK(cudaMemcpy(plan->maps, maps.data(), mb, cudaMemcpyHostToDevice));
    return NL_OK;
}

nl_status lu_grouped_plan(int count, const GInst* host_inst, int nb, int gemm, bool fp64, GroupPlan* plan, int kind,
                          int tm)
{
    if (count < 1 || nb < 16 || nb > 128 || nb % 16) {
        set_error("grouped LU: need count >= 1 and nb a multiple of 16 in [16, 128]");
        return NL_EINVAL;
    }
    if (kind == 1) {
        if (fp64 || !(gemm == 1 || gemm == 2) || nb > 64 || (gemm == 2 && nb != 64) || !(tm == 64 || tm == 128) ||
            !tc_gemm_supported() || !tc_error_word()) {
            set_error("grouped LU: the persistent launch needs the binary16 LU, nb <= 64 (nb = 64 with the "
                      "tensor-core update), SIMT tile height 64 or 128");
            return NL_EINVAL;
        }
        return lu_grouped_plan_p(count, host_inst, nb, gemm, tm, plan);
    }
    if (kind != 0) {
        set_error("grouped LU: unknown kind %d", kind);
        return NL_EINVAL;
    }
    if (fp64) gemm = 1;
    if (gemm == 2 && (nb % 64 || !tc_gemm_supported())) gemm = 1;
    int nmax = 0;
    for (int i = 0; i < count; ++i) nmax = std::max(nmax, host_inst[i].N);
    // largest matrices first in every task list
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return host_inst[a].N > host_inst[b].N; });
    const int steps = (int)cdiv(nmax, nb);
    const int rows_per_cta = fp64 ? kOffThreads / kOffG : kO16Rows;
    const int tile = (gemm == 2) ? 128 : 64;
    std::vector<GTask> tasks;
    plan->off.assign(3 * steps, 0);
    plan->n.assign(3 * steps, 0);
    for (int k = 0; k < steps; ++k) {
        const int K = k * nb;
        plan->off[3 * k] = (int)tasks.size();
        for (int i : order)
            if (host_inst[i].N > K) tasks.push_back({i, 0, 0, 0});
        plan->n[3 * k] = (int)tasks.size() - plan->off[3 * k];
        plan->off[3 * k + 1] = (int)tasks.size();
        for (int i : order) {
            const int rest = host_inst[i].N - K - nb;
            if (rest <= 0) continue;
            const int nrb = (int)cdiv(rest, rows_per_cta);
            for (int b = 0; b < 2 * nrb; ++b) tasks.push_back({i, b, nrb, 0});
        }
        plan->n[3 * k + 1] = (int)tasks.size() - plan->off[3 * k + 1];
        plan->off[3 * k + 2] = (int)tasks.size();
        for (int i : order) {
            const int rest = host_inst[i].N - K - nb;
            if (rest <= 0) continue;
            const int nt = (int)cdiv(rest, tile);
            for (int a = 0; a < nt; ++a)
                for (int b = 0; b < nt; ++b) tasks.push_back({i, a * tile, b * tile, 0});
        }
        plan->n[3 * k + 2] = (int)tasks.size() - plan->off[3 * k + 2];
    }
    lu_grouped_free(plan);
    plan->count = count;
    plan->nb = nb;
    plan->gemm = gemm;
    plan->steps = steps;
    plan->fp64 = fp64;
    std::vector<TmapBytes> maps;
    if (gemm == 2) {
        maps.resize(2 * (size_t)count);
        for (int i = 0; i < count; ++i)
            if (host_inst[i].N > nb && !tc_encode_instance_maps(reinterpret_cast<const __half*>(host_inst[i].A), host_inst[i].N,
                                         host_inst[i].ld, host_inst[i].ut, nb, &maps[2 * (size_t)i])) {
                set_error("grouped LU: tensor-map encoding failed for matrix %d", i);
                return NL_ECUDA;
            }
    }
    const size_t tb = tasks.size() * sizeof(GTask), mb = maps.size() * sizeof(TmapBytes);
    plan->bytes = round_up(tb, 256) + mb + 256;
    void* p = nullptr;
    NL_CUDA_OK(cudaMalloc(&p, plan->bytes));
    plan->tasks = reinterpret_cast<GTask*>(p);
    plan->maps = mb ? reinterpret_cast<TmapBytes*>((char*)p + round_up(tb, 256)) : nullptr;
    if (tb) NL_CUDA_OK(cudaMemcpy(plan->tasks, tasks.data(), tb, cudaMemcpyHostToDevice));
    if (mb) NL_CUDA_OK(cudaMemcpy(plan->maps, maps.data(), mb, cudaMemcpyHostToDevice));
    return NL_OK;
}

void lu_grouped_free(GroupPlan* plan)
{
    if (plan->tasks) cudaFree(plan->tasks);
    plan->tasks = nullptr;
    plan->maps = nullptr;
    plan->ptasks = nullptr;
    plan->ctl = nullptr;
    plan->nptasks = 0;
    plan->kind = 0;
}

nl_status lu_grouped_setup()
{
    static bool smem_set = false;
    if (!smem_set) {
        if (set_max_dynamic_smem((const void*)k_diag_lu16_g) != NL_OK ||
            set_max_dynamic_smem((const void*)k_offdiag16_g) != NL_OK ||
            set_max_dynamic_smem((const void*)k_diag_lu_g<double, double, false>) != NL_OK ||
            set_max_dynamic_smem((const void*)k_offdiag_g<double, double, false>) != NL_OK ||
            set_max_dynamic_smem((const void*)k_lu_grouped_p<false>) != NL_OK ||
            set_max_dynamic_smem((const void*)k_lu_grouped_p<true>) != NL_OK)
            return NL_ECUDA;
        smem_set = true;
    }
    return NL_OK;
}

nl_status lu_grouped_factor(const GroupPlan& plan, const GInst* dev_inst, cudaStream_t st, int* launches)
{
    NL_TRY(lu_grouped_setup());
    const int nb = plan.nb, wp = (int)round_up(nb, 32);
    if (plan.kind == 1) {
        k_pg_init<<<1, 256, 0, st>>>(plan.ctl, plan.count, dev_inst);  // a kernel node: legal in conditional bodies
        prof_begin("k_lu_grouped_p", st);
        unsigned long long* ts = pg_task_stats_ptr();
        if (plan.gemm == 2)
            k_lu_grouped_p<true><<<plan.grid, kPgThreads, pg_smem_bytes(nb), st>>>(
                plan.ptasks, plan.nptasks, nb, plan.tm, plan.tn, plan.maps, plan.ctl, plan.count, tc_error_word(),
                ts);
        else
            k_lu_grouped_p<false><<<plan.grid, kPgThreads, pg_smem_bytes(nb), st>>>(
                plan.ptasks, plan.nptasks, nb, plan.tm, plan.tn, nullptr, plan.ctl, plan.count, tc_error_word(),
                ts);
        prof_end("k_lu_grouped_p", st);
        NL_CUDA_OK(cudaGetLastError());
        if (launches) *launches += 2;
        return NL_OK;
    }
    int nl = 0;
    for (int k = 0; k < plan.steps; ++k) {
        const int K = k * nb;
        const GTask* td = plan.tasks + plan.off[3 * k];
        const GTask* to = plan.tasks + plan.off[3 * k + 1];
        const GTask* tg = plan.tasks + plan.off[3 * k + 2];
        const int nd = plan.n[3 * k], no = plan.n[3 * k + 1], ng = plan.n[3 * k + 2];
        if (plan.fp64) {
            if (nd) {
                prof_begin("k_diag_lu", st);
                k_diag_lu_g<double, double, false><<<nd, kDiagThreads, (size_t)wp * (wp + 1) * 8, st>>>(dev_inst, td,
                                                                                                      K, nb);
                prof_end("k_diag_lu", st);
            }
            if (no) {
                prof_begin("k_offdiag", st);
                k_offdiag_g<double, double, false><<<no, kOffThreads,
                                                     (size_t)wp * wp * 8 + (size_t)wp * (kOffThreads / kOffG) * 8,
                                                     st>>>(dev_inst, to, K, nb);
                prof_end("k_offdiag", st);
            }
            if (ng) k_gemm_simt_g<double, double><<<ng, 256, 0, st>>>(dev_inst, tg, K, nb);
        } else {
            if (nd) {
                prof_begin("k_diag_lu16", st);
                k_diag_lu16_g<<<nd, kD16Threads, kDiag16Smem, st>>>(dev_inst, td, K, nb);
                prof_end("k_diag_lu16", st);
            }
            if (no) {
                prof_begin("k_offdiag16", st);
                k_offdiag16_g<<<no, kO16Threads, offdiag16_smem(wp), st>>>(dev_inst, to, K, nb, plan.gemm == 2);
                prof_end("k_offdiag16", st);
            }
            if (ng) {
                if (plan.gemm == 2) {
                    nl_status s = tc_gemm16_grouped(dev_inst, plan.maps, tg, ng, K, nb, st);
                    if (s != NL_OK) return s;
                } else {
                    k_gemm_simt_g<__half, float><<<ng, 256, 0, st>>>(dev_inst, tg, K, nb);
                }
            }
        }
        nl += (nd > 0) + (no > 0) + (ng > 0);
        NL_CUDA_OK(cudaGetLastError());
    }
    if (launches) *launches += nl;
    return NL_OK;
}

// The multiplier rounding of the binary16 LU, elementwise (for tests).
__global__ void k_div_round16(int64_t n, const float* __restrict__ a, const float* __restrict__ b,
                              float* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = div_round_h(a[i], b[i], __frcp_rn(b[i]));
}

}  // namespace nl

extern "C" nl_status nl_k_div_round16(int64_t n, const float* a, const float* b, float* out, void* stream)
{
    using namespace nl;
    if (n < 0 || (n > 0 && (!a || !b || !out))) {
        set_error("nl_k_div_round16: bad argument");
        return NL_EINVAL;
    }
    if (n == 0) return NL_OK;
    k_div_round16<<<(unsigned)cdiv(n, 256), 256, 0, (cudaStream_t)stream>>>(n, a, b, out);
    NL_CUDA_OK(cudaGetLastError());
    return NL_OK;
}

extern "C" nl_status nl_debug_grouped_task_times(int enable, double* out9)
{
    using namespace nl;
    unsigned long long v[9] = {};
    NL_CUDA_OK(cudaDeviceSynchronize());
    NL_CUDA_OK(cudaMemcpyFromSymbol(v, g_pg_tstat, sizeof(v)));
    const unsigned long long z[9] = {};
    NL_CUDA_OK(cudaMemcpyToSymbol(g_pg_tstat, z, sizeof(z)));
    int dev = 0, khz = 0;
    NL_CUDA_OK(cudaGetDevice(&dev));
    NL_CUDA_OK(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
    if (out9)
        for (int k = 0; k < 3; ++k) {
            out9[3 * k] = (double)v[3 * k];
            out9[3 * k + 1] = khz > 0 ? (double)v[3 * k + 1] / (khz * 1e-3) : 0.0;  // cycles -> microseconds
            out9[3 * k + 2] = khz > 0 ? (double)v[3 * k + 2] / (khz * 1e-3) : 0.0;
        }
    g_pg_tstat_on.store(enable != 0);
    return NL_OK;
}

extern "C" nl_status nl_debug_grouped_wait_limit(long long polls)
{
    using namespace nl;
    NL_CUDA_OK(cudaMemcpyToSymbol(g_pg_spin_limit, &polls, sizeof(polls)));
    return NL_OK;
}
