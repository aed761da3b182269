// batch.cu — many independent H-equation solves (Section 3, eq. (3.2)) of
// different N and c, advanced together: every Newton step of every instance
// runs in grouped launches (one launch per kernel class covers all
// instances), and the whole solve is one CUDA graph with two conditional
// WHILE nodes, so the host waits once per batch instead of once per step.
//
//   init: x = x0, F(x), tau = tol ||F(x0)|| + tau_a          (Algorithm 1.1)
//   WHILE some instance is active:                            (Newton)
//     J32 and J16 (or J64) at x                                (Sections 1.1, 3)
//     grouped LU of J16 (no interchanges; an instance that would need one
//       leaves the batch), b = fl32(-F/||F||), u = 0           (eq. (2.17))
//     WHILE some instance's IR continues:                      (Algorithm IR)
//       u += U^{-1} L^{-1} r;  r = b - J32 u;  test eta / failure / cap
//     x <- x + ||F|| u and F(x), then the termination test     (eq. (2.18))
//
// Mode IR16 with fallback: an instance whose IR stalls (the failure rule of
// Section 3.1 fires, or the cap is reached without meeting eta) leaves the
// batch at that step; the host finishes it on the single-instance path with
// GMRES-IR (Section 2.2), which redoes that step.  The same happens, in the
// batch's mode, to an instance whose factorisation needs row interchanges.
// FP64 mode: J64, the grouped double LU and one direct solve per step.
//
// Every loop in the graph is bounded: each conditional kernel stops its loop
// after the configured cap.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace nl {

constexpr int kBtThreads = 512;  // grouped triangular solve: one CTA per instance
constexpr int kBMaxN = 8192;     // batch instances keep their vector in shared memory
// Instances are grouped by N into buckets (N <= 128, 129..256, ..., 4097..8192),
// each factored by its own grouped LU on its own stream.
constexpr int kBMaxBuckets = 7;
constexpr int kBucketNmax[kBMaxBuckets] = {128, 256, 512, 1024, 2048, 4096, 8192};

struct BCtl {
    int lin_count, act_count, ir_round, newton_round;
    int ir_total, pad[3];
};

struct BParams {  // per-solve scalars read by the graph
    double tol, tau_a;
};

// ------------------------------------------------------------ device side --

// 32 consecutive factor entries p[0..31] of one row into registers as T;
// entries at or past `valid` read as zero.
template <typename S, typename T>
__device__ __forceinline__ void load_seg32(const S* __restrict__ p, int valid, bool vec, T* out)
{
    if (vec && valid >= 32) {
        constexpr int V = 16 / sizeof(S);
#pragma unroll
        for (int q = 0; q < 32 / V; ++q) {
            const uint4 raw = reinterpret_cast<const uint4*>(p)[q];
            const S* e = reinterpret_cast<const S*>(&raw);
#pragma unroll
            for (int k = 0; k < V; ++k) out[q * V + k] = (T)ld_elem(e + k);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) out[j] = (j < valid) ? (T)ld_elem(p + j) : T(0);
    }
}

// 8 consecutive entries (the caller's 8-column group) of one row.
template <typename S, typename T>
__device__ __forceinline__ void load_seg8(const S* __restrict__ p, int valid, bool vec, T* out)
{
    if (vec && valid >= 8) {
        constexpr int V = 16 / sizeof(S);
#pragma unroll
        for (int q = 0; q < 8 / V; ++q) {
            const uint4 raw = reinterpret_cast<const uint4*>(p)[q];
            const S* e = reinterpret_cast<const S*>(&raw);
#pragma unroll
            for (int k = 0; k < V; ++k) out[q * V + k] = (T)ld_elem(e + k);
        }
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) out[k] = (k < valid) ? (T)ld_elem(p + k) : T(0);
    }
}

// y <- U^{-1} L^{-1} y in place (y in shared memory, N entries) with the
// factors of an LU without interchanges (unit lower L below the diagonal, U
// on and above it), factor entries promoted to T on load (eq. (2.16)).
// Blocks of 32 rows: warp 0 substitutes within the diagonal block (lane i =
// row i, shuffle broadcasts), then all warps apply the block's contribution
// to the rows still to be solved (four lanes per row, eight columns each).
template <typename S, typename T>
__device__ void trsv_core(int N, const S* __restrict__ LU, int64_t ld, T* y)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = kBtThreads / 32;
    const bool vec = ((((uintptr_t)LU) & 15) == 0) && ((ld * (int64_t)sizeof(S)) % 16 == 0);
    const int nblk = (N + 31) / 32;
    const int q = lane & 3;
    for (int b = 0; b < nblk; ++b) {
        const int r0 = 32 * b, nb_ = min(32, N - r0);
        if (warp == 0) {
            const int i = lane;
            T yi = (i < nb_) ? y[r0 + i] : T(0);
            T Lr[32];
            // entries at and right of the diagonal are loaded but never used (t < i below)
            load_seg32<S, T>(LU + (int64_t)(r0 + min(i, nb_ - 1)) * ld + r0, (i < nb_) ? nb_ : 0,
                             vec && nb_ == 32, Lr);
#pragma unroll
            for (int t = 0; t < 32; ++t) {
                const T yt = __shfl_sync(0xffffffffu, yi, t);
                if (t < i) yi = fma(-Lr[t], yt, yi);
            }
            if (i < nb_) y[r0 + i] = yi;
        }
        __syncthreads();
        if (r0 + 32 < N) {
            T yq[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) yq[e] = y[r0 + 8 * q + e];
            for (int ib = r0 + 32 + warp * 8; ib < N; ib += NW * 8) {
                const int i = ib + (lane >> 2);
                const bool ok = i < N;
                T l[8];
                load_seg8<S, T>(LU + (int64_t)(ok ? i : ib) * ld + r0 + 8 * q, ok ? 8 : 0, vec, l);
                T s = T(0);
#pragma unroll
                for (int e = 0; e < 8; ++e) s = fma(l[e], yq[e], s);
                s += __shfl_xor_sync(0xffffffffu, s, 1);
                s += __shfl_xor_sync(0xffffffffu, s, 2);
                if (ok && q == 0) y[i] -= s;
            }
        }
        __syncthreads();
    }
    for (int b = nblk - 1; b >= 0; --b) {
        const int r0 = 32 * b, nb_ = min(32, N - r0);
        if (warp == 0) {
            const int i = lane;
            T zi = (i < nb_) ? y[r0 + i] : T(0);
            T Ur[32];
            load_seg32<S, T>(LU + (int64_t)(r0 + min(i, nb_ - 1)) * ld + r0, (i < nb_) ? nb_ : 0,
                             vec && nb_ == 32, Ur);
#pragma unroll
            for (int t = 31; t >= 0; --t) {
                if (t < nb_) {
                    if (i == t) zi = zi / Ur[t];
                    const T zt = __shfl_sync(0xffffffffu, zi, t);
                    if (i < t) zi = fma(-Ur[t], zt, zi);
                }
            }
            if (i < nb_) y[r0 + i] = zi;
        }
        __syncthreads();
        if (r0 > 0) {
            T zq[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) zq[e] = (8 * q + e < nb_) ? y[r0 + 8 * q + e] : T(0);
            const int valid = max(0, min(8, nb_ - 8 * q));
            for (int ib = warp * 8; ib < r0; ib += NW * 8) {
                const int i = ib + (lane >> 2);
                const bool ok = i < r0;
                T u[8];
                load_seg8<S, T>(LU + (int64_t)(ok ? i : ib) * ld + r0 + 8 * q, ok ? valid : 0, vec, u);
                T s = T(0);
#pragma unroll
                for (int e = 0; e < 8; ++e) s = fma(u[e], zq[e], s);
                s += __shfl_xor_sync(0xffffffffu, s, 1);
                s += __shfl_xor_sync(0xffffffffu, s, 2);
                if (ok && q == 0) y[i] -= s;
            }
        }
        __syncthreads();
    }
}

// Batch correction: d = U^{-1} L^{-1} r and u += d (IR, binary16 factors), or
// u64 = U^{-1} L^{-1} b64 (FP64 mode).  One CTA per instance, largest first.
template <typename S, typename T>
__global__ void __launch_bounds__(kBtThreads) k_b_trsv(const BInst* __restrict__ inst, const BState* __restrict__ st,
                                                       const int* __restrict__ order)
{
    extern __shared__ __align__(16) unsigned char bt_smem[];
    T* y = reinterpret_cast<T*>(bt_smem);
    constexpr bool kDirect = std::is_same<S, double>::value;
    const int id = order[blockIdx.x];
    const BInst& I = inst[id];
    const BState& S_ = st[id];
    if (S_.status != BS_ACTIVE || (!kDirect && !S_.lin_active)) return;
    const int N = I.N;
    const T* rhs;
    if constexpr (kDirect) rhs = I.b64;
    else rhs = I.r;
    for (int i = threadIdx.x; i < N; i += kBtThreads) y[i] = rhs[i];
    __syncthreads();
    trsv_core<S, T>(N, reinterpret_cast<const S*>(I.J), I.ld, y);
    if constexpr (kDirect) {
        for (int i = threadIdx.x; i < N; i += kBtThreads) I.u64[i] = y[i];
    } else {
        for (int i = threadIdx.x; i < N; i += kBtThreads) I.u[i] = I.u[i] + y[i];
    }
}

// Kernel-level grouped solve b <- U^{-1} L^{-1} P b with LAPACK-style ipiv.
struct GSolve {
    const void* LU;
    int64_t ld;
    int N, pad;
    const int* ipiv;
    void* b;
};

template <typename S, typename T>
__global__ void __launch_bounds__(kBtThreads) k_trsv_grouped(const GSolve* __restrict__ items)
{
    extern __shared__ __align__(16) unsigned char bt_smem[];
    T* y = reinterpret_cast<T*>(bt_smem);
    const GSolve it = items[blockIdx.x];
    const int N = it.N;
    T* b = reinterpret_cast<T*>(it.b);
    bool swaps = false;
    for (int i = threadIdx.x; i < N; i += kBtThreads) {
        y[i] = b[i];
        swaps |= (it.ipiv[i] != i);
    }
    if (__syncthreads_or(swaps) && threadIdx.x == 0) {
        for (int k = 0; k < N; ++k) {
            const int p = it.ipiv[k];
            if (p != k && p >= 0 && p < N) {
                const T t = y[k];
                y[k] = y[p];
                y[p] = t;
            }
        }
    }
    __syncthreads();
    trsv_core<S, T>(N, reinterpret_cast<const S*>(it.LU), it.ld, y);
    for (int i = threadIdx.x; i < N; i += kBtThreads) b[i] = y[i];
}

// x[0] = x0 (ones when x0 is NULL) and a fresh state for every instance.
__global__ void __launch_bounds__(256) k_b_init(const BInst* __restrict__ inst, BState* __restrict__ st)
{
    const BInst& I = inst[blockIdx.x];
    for (int i = threadIdx.x; i < I.N; i += blockDim.x) I.x[0][i] = I.x0 ? I.x0[i] : 1.0;
    if (threadIdx.x == 0) {
        BState s;
        memset(&s, 0, sizeof(s));
        st[blockIdx.x] = s;
        I.cnt[0] = 0u;
        I.cnt[1] = 0u;
    }
}

// After F(x0): ||F(x0)||, tau, the first decision (Algorithm 1.1).
__global__ void __launch_bounds__(256) k_b_init_check(const BInst* __restrict__ inst, BState* __restrict__ st,
                                                      int count, const BParams* __restrict__ prm, int newton_maxit,
                                                      double* __restrict__ hist, BCtl* __restrict__ ctl)
{
    const double tol = prm->tol, tau_a = prm->tau_a;
    int act = 0;
    for (int k = threadIdx.x; k < count; k += blockDim.x) {
        BState& S = st[k];
        S.fn0 = S.fn;
        S.tau = tol * S.fn0 + tau_a;
        hist[(size_t)k * NL_MAX_HIST] = 1.0;
        int s = BS_ACTIVE;
        if (S.fn <= S.tau) s = BS_CONVERGED;
        else if (!isfinite(S.fn)) s = BS_NUMERIC;
        else if (newton_maxit <= 0) s = BS_NOTCONV;
        S.status = s;
        *inst[k].flag = (s == BS_ACTIVE) ? 0 : 2;
        act += (s == BS_ACTIVE);
    }
    if (act) atomicAdd(&ctl->act_count, act);
}

// Sets a WHILE node's condition: continue while some instance is still in
// the loop and the loop has run fewer than `cap` times.
__global__ void k_b_cond(BCtl* __restrict__ ctl, int which, int reset, int cap, cudaGraphConditionalHandle h)
{
    int* count = which ? &ctl->lin_count : &ctl->act_count;
    int* round = which ? &ctl->ir_round : &ctl->newton_round;
    if (reset) *round = 0;
    const unsigned v = (*count > 0 && *round < cap) ? 1u : 0u;
    if (v) {
        *round += 1;
        if (which) ctl->ir_total += 1;
    }
    *count = 0;
    cudaGraphSetConditional(h, v);
}

// After the grouped LU: park instances whose factorisation needs row
// interchanges; form b = fl32(-F/||F||) (eq. (2.17)), r = b, u = 0,
// ||b|| and the IR state (Algorithm IR, u0 = 0).
__global__ void __launch_bounds__(256) k_b_rhs(const BInst* __restrict__ inst, BState* __restrict__ st, double eta,
                                               int maxit, int park_all, BCtl* __restrict__ ctl)
{
    __shared__ double red[8];
    const BInst& I = inst[blockIdx.x];
    BState& S = st[blockIdx.x];
    if (S.status != BS_ACTIVE) return;
    if (park_all || (*(volatile int*)I.flag & 1)) {
        if (threadIdx.x == 0) S.status = BS_PARKED_LU;
        return;
    }
    const double fn = S.fn;
    double s = 0.0;
    for (int i = threadIdx.x; i < I.N; i += blockDim.x) {
        const float bi = (float)(-I.F[i] / fn);
        I.b[i] = bi;
        I.r[i] = bi;
        I.u[i] = 0.0f;
        s += (double)bi * (double)bi;
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) {
        const double nb = sqrt(s);
        S.nb = nb;
        S.nr = nb;
        S.prev = nb;
        S.outer = 0;
        S.lin_iters = 0;
        S.failed = 0;
        const bool conv = nb <= eta * nb;
        S.lin_active = (!conv && maxit > 0) ? 1 : 0;
        if (!conv && !S.lin_active) S.status = BS_PARKED_IR;
        if (S.lin_active) atomicAdd(&ctl->lin_count, 1);
    }
}

__global__ void __launch_bounds__(256) k_b_rhs64(const BInst* __restrict__ inst, BState* __restrict__ st,
                                                 int park_all)
{
    const BInst& I = inst[blockIdx.x];
    BState& S = st[blockIdx.x];
    if (S.status != BS_ACTIVE) return;
    if (park_all || (*(volatile int*)I.flag & 1)) {
        if (threadIdx.x == 0) S.status = BS_PARKED_LU;
        return;
    }
    const double fn = S.fn;
    for (int i = threadIdx.x; i < I.N; i += blockDim.x) I.b64[i] = -I.F[i] / fn;
}

// After r = b - J32 u: the IR tests of Section 3.1.  Success at
// ||r|| <= eta ||b||; the failure rule (the residual norm grew) or the cap
// without success is a stall, and the instance leaves the batch.
__global__ void __launch_bounds__(256) k_b_ir_check(BState* __restrict__ st, int count, double eta, int maxit,
                                                    BCtl* __restrict__ ctl)
{
    int act = 0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
        BState& S = st[k];
        if (S.status != BS_ACTIVE || !S.lin_active) continue;
        S.outer += 1;
        S.lin_iters += 1;
        const double nr = S.nr_new;
        if (nr > S.prev) {
            S.failed = 1;
            S.lin_active = 0;
            S.status = BS_PARKED_IR;
            continue;
        }
        S.prev = nr;
        S.nr = nr;
        if (nr <= eta * S.nb) {
            S.lin_active = 0;
        } else if (S.outer >= maxit) {
            S.lin_active = 0;
            S.status = BS_PARKED_IR;
        } else {
            ++act;
        }
    }
    if (act) atomicAdd(&ctl->lin_count, act);
}

// After x <- x + ||F|| u and F(x): step bookkeeping and the termination
// test of Algorithm 1.1; the flags of the next factorisation.
__global__ void __launch_bounds__(256) k_b_newton_check(const BInst* __restrict__ inst, BState* __restrict__ st,
                                                        int count, int newton_maxit, int fp64,
                                                        double* __restrict__ hist, int* __restrict__ lin_iters,
                                                        int* __restrict__ lin_outer, int* __restrict__ lin_failed,
                                                        double* __restrict__ lin_relres, BCtl* __restrict__ ctl)
{
    int act = 0;
    for (int k = threadIdx.x; k < count; k += blockDim.x) {
        BState& S = st[k];
        if (S.status != BS_ACTIVE) {
            *inst[k].flag = 2;
            continue;
        }
        const size_t h = (size_t)k * NL_MAX_HIST;
        if (!fp64) {
            lin_iters[h + S.it] = S.lin_iters;
            lin_outer[h + S.it] = S.outer;
            lin_failed[h + S.it] = S.failed;
            lin_relres[h + S.it] = S.nb > 0.0 ? S.nr / S.nb : 0.0;
        }
        S.it += 1;
        S.par ^= 1;
        hist[h + S.it] = S.fn0 > 0.0 ? S.fn / S.fn0 : 0.0;
        int s = BS_ACTIVE;
        if (S.fn <= S.tau) s = BS_CONVERGED;
        else if (!isfinite(S.fn)) s = BS_NUMERIC;
        else if (S.it >= newton_maxit) s = BS_NOTCONV;
        S.status = s;
        *inst[k].flag = (s == BS_ACTIVE) ? 0 : 2;
        act += (s == BS_ACTIVE);
    }
    if (act) atomicAdd(&ctl->act_count, act);
}

// The current iterate of every instance into the packed output.
__global__ void __launch_bounds__(256) k_b_gather(const BInst* __restrict__ inst, const BState* __restrict__ st)
{
    const BInst& I = inst[blockIdx.x];
    const double* x = I.x[st[blockIdx.x].par];
    for (int i = threadIdx.x; i < I.N; i += blockDim.x) I.xout[i] = x[i];
}

__global__ void k_b_fill(int64_t n, double v, double* x)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

__global__ void k_htab_g(int n, double* htab, float* htab32)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) {
        const double h = 1.0 / (double)(k + 1);
        htab[k] = h;
        htab32[k] = (float)h;
    }
}

// --------------------------------------------------------------- host side --

// Appends a WHILE node controlled by h to the graph that `s` is capturing,
// after everything captured so far, and starts capturing its body on
// `body_stream`.  h must belong to that graph.
static nl_status add_while_node(cudaStream_t s, cudaStream_t body_stream, cudaGraphConditionalHandle h)
{
    cudaStreamCaptureStatus cs;
    cudaGraph_t g;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    NL_CUDA_OK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    NL_CUDA_OK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &p));
    NL_CUDA_OK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    NL_CUDA_OK(cudaStreamBeginCaptureToGraph(body_stream, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                             cudaStreamCaptureModeRelaxed));
    return NL_OK;
}

nl_status batch_trsv_smem_setup()
{
    static bool done = false;
    if (done) return NL_OK;
    if (set_max_dynamic_smem((const void*)k_b_trsv<__half, float>) != NL_OK ||
        set_max_dynamic_smem((const void*)k_b_trsv<double, double>) != NL_OK ||
        set_max_dynamic_smem((const void*)k_trsv_grouped<__half, float>) != NL_OK ||
        set_max_dynamic_smem((const void*)k_trsv_grouped<double, double>) != NL_OK)
        return NL_ECUDA;
    done = true;
    return NL_OK;
}

}  // namespace nl

using namespace nl;

struct nl_batch {
    int count = 0;
    nl_config cfg;
    std::vector<int> N;
    std::vector<double> c;
    std::vector<int64_t> off;  // packed vector offsets
    std::vector<int> ld;
    int nmax = 0, total_rows = 0;
    cudaStream_t st = nullptr, s1 = nullptr, s2 = nullptr;
    bool own_streams = false, own_st = true;
    // device memory
    void* pool = nullptr;
    size_t pool_bytes = 0;
    void* pool64 = nullptr;
    size_t pool64_bytes = 0;
    BInst* dinst = nullptr;       // three-precision table
    BInst* dinst64 = nullptr;     // FP64 table (J = J64)
    std::vector<BInst> hinst, hinst64;
    BState* dst = nullptr;
    BCtl* ctl = nullptr;
    BParams* prm = nullptr;
    int* flags = nullptr;
    GInst* gin = nullptr;         // grouped-LU tables (binary16 and double)
    GInst* gin64 = nullptr;
    std::vector<GInst> hgin, hgin64;
    BTask *res_tasks = nullptr, *gemv_tasks = nullptr;
    int n_res = 0, n_gemv = 0;
    int* row_off = nullptr;
    int* order = nullptr;
    double* htab = nullptr;
    float* htab32 = nullptr;  // the same table rounded to single (the Jacobian's entries use it)
    double *x0 = nullptr, *xout = nullptr;
    double* hist = nullptr;
    int *lin_iters = nullptr, *lin_outer = nullptr, *lin_failed = nullptr;
    double* lin_relres = nullptr;
    GroupPlan plan64;
    int nb = 128, gemm = 2;       // the choice of the bucket that holds the largest instance
    // N buckets of the binary16 grouped LU, factored side by side on their own streams,
    // each with its own outer block and update (autotuned per bucket)
    int nbk = 0;
    int bk_nmax[kBMaxBuckets] = {}, bk_count[kBMaxBuckets] = {}, bk_nb[kBMaxBuckets] = {},
        bk_gemm[kBMaxBuckets] = {}, bk_cached[kBMaxBuckets] = {}, bk_id[kBMaxBuckets] = {};
    std::vector<int> bk_of;                     // bucket of each instance
    std::vector<std::vector<GInst>> bk_hgin;    // host copies of the bucket tables
    GInst* bk_gin[kBMaxBuckets] = {};           // device bucket tables (in the pool)
    GroupPlan bk_plan[kBMaxBuckets];
    cudaStream_t bk_st[kBMaxBuckets] = {};
    cudaEvent_t bk_ev[kBMaxBuckets] = {}, ev_fork = nullptr;
    // graphs (built on first use per mode)
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    int nodes_init = 0, nodes_newton[2] = {0, 0}, nodes_ir = 0;
    // results
    std::vector<nl_stats_t> stats;
    nl_batch_info_t info;
    // autotuning record
    std::vector<int> tune_nb, tune_gemm, tune_bucket;
    std::vector<double> tune_ms;
    // last solve
    std::vector<BState> hstate;
    std::vector<nl_stats_t> single;
    std::vector<int> single_used;
    bool stats_ready = false;
    int last_fp64 = 0;
};

static nl_status batch_build_graph(nl_batch* B, int fp64);

static void batch_free(nl_batch* B)
{
    if (!B) return;
    if (B->st) cudaStreamSynchronize(B->st);
    for (int m = 0; m < 2; ++m)
        if (B->exec[m]) cudaGraphExecDestroy(B->exec[m]);
    for (int b = 0; b < kBMaxBuckets; ++b) {
        lu_grouped_free(&B->bk_plan[b]);
        if (B->bk_st[b]) cudaStreamDestroy(B->bk_st[b]);
        if (B->bk_ev[b]) cudaEventDestroy(B->bk_ev[b]);
    }
    if (B->ev_fork) cudaEventDestroy(B->ev_fork);
    lu_grouped_free(&B->plan64);
    if (B->pool) cudaFree(B->pool);
    if (B->pool64) cudaFree(B->pool64);
    if (B->own_streams) {
        if (B->st && B->own_st) cudaStreamDestroy(B->st);
        if (B->s1) cudaStreamDestroy(B->s1);
        if (B->s2) cudaStreamDestroy(B->s2);
    }
    delete B;
}

// The binary16 grouped-LU plan of bucket b for outer block nb and update g
// (1 SIMT and 2 tcgen05, three launches per outer step; 3 / 4 one persistent
// launch with 64 x 64 / 128 x 64 SIMT update tiles, 5 one persistent launch
// with 128 x 128 tcgen05 update tiles).
static nl_status batch_plan16(nl_batch* B, int b, int nb, int g, GroupPlan* pl)
{
    const int n = B->bk_count[b];
    const GInst* h = B->bk_hgin[b].data();
    if (g == 5) return lu_grouped_plan(n, h, nb, 2, false, pl, 1, 128);
    if (g >= 3) return lu_grouped_plan(n, h, nb, 1, false, pl, 1, g == 3 ? 64 : 128);
    return lu_grouped_plan(n, h, nb, g, false, pl);
}

// The binary16 grouped LU of every bucket: one bucket on the given stream, or
// a fork to the buckets' streams and a join back (stream-capturable).
static nl_status batch_lu16(nl_batch* B, cudaStream_t st, int* launches)
{
    if (B->nbk == 1) return lu_grouped_factor(B->bk_plan[0], B->bk_gin[0], st, launches);
    NL_CUDA_OK(cudaEventRecord(B->ev_fork, st));
    for (int b = 0; b < B->nbk; ++b) {
        NL_CUDA_OK(cudaStreamWaitEvent(B->bk_st[b], B->ev_fork, 0));
        NL_TRY(lu_grouped_factor(B->bk_plan[b], B->bk_gin[b], B->bk_st[b], launches));
        NL_CUDA_OK(cudaEventRecord(B->bk_ev[b], B->bk_st[b]));
        NL_CUDA_OK(cudaStreamWaitEvent(st, B->bk_ev[b], 0));
    }
    return NL_OK;
}

// Device time of one whole grouped LU (all buckets) on the Jacobians at
// x0 = ones, best of three.
static nl_status batch_time_lu16(nl_batch* B, double* ms_out)
{
    cudaEvent_t e0, e1;
    NL_CUDA_OK(cudaEventCreate(&e0));
    NL_CUDA_OK(cudaEventCreate(&e1));
    k_b_init<<<B->count, 256, 0, B->st>>>(B->dinst, B->dst);
    nl_status s = launch_residual_g(B->dinst, B->dst, B->res_tasks, B->n_res, 0, B->htab, B->st);
    float best = 1e30f;
    for (int rep = 0; rep < 3 && s == NL_OK; ++rep) {
        if (cudaMemsetAsync(B->flags, 0, sizeof(int) * B->count, B->st) != cudaSuccess) s = NL_ECUDA;
        if (s == NL_OK)
            s = launch_jacobian_g(B->dinst, B->dst, B->row_off, B->count, B->total_rows, B->htab, B->htab32, 0,
                                  B->st);
        if (s != NL_OK) break;
        cudaEventRecord(e0, B->st);
        s = batch_lu16(B, B->st, nullptr);
        cudaEventRecord(e1, B->st);
        if (s == NL_OK && cudaEventSynchronize(e1) != cudaSuccess) s = NL_ECUDA;
        float ms = 0.0f;
        if (s == NL_OK) cudaEventElapsedTime(&ms, e0, e1);
        best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_out = s == NL_OK ? best : 0.0;
    return s;
}

// ---- the tuning table: a JSON file (path in the environment variable
// NL_LU_TUNE_FILE) that keeps each bucket's choice between processes, one
// entry per line:  "<key>": {"nb": 64, "gemm": 2, "ms": 1.234}
// keyed by device, SM count, bucket range and instance count (next power of two).
static std::string tune_key(const nl_batch* B, int b)
{
    int dev = 0, nsm = num_sms();
    cudaGetDevice(&dev);
    cudaDeviceProp pr;
    std::string name = cudaGetDeviceProperties(&pr, dev) == cudaSuccess ? pr.name : "unknown";
    for (char& ch : name)
        if (ch == '"' || ch == '\\' || ch == '\n') ch = '_';
    int cp = 1;
    while (cp < B->bk_count[b]) cp *= 2;
    const int id = B->bk_id[b], lo = id ? kBucketNmax[id - 1] + 1 : 1;
    char buf[256];
    snprintf(buf, sizeof buf, "%s|sm%d|N%d-%d|count%d", name.c_str(), nsm, lo, kBucketNmax[id], cp);
    return buf;
}

struct TuneEntry {
    int nb = 0, gemm = 0;
    double ms = 0.0;
};

static std::map<std::string, TuneEntry> tune_read(const char* path)
{
    std::map<std::string, TuneEntry> m;
    FILE* f = path ? fopen(path, "r") : nullptr;
    if (!f) return m;
    char line[1024];
    while (fgets(line, sizeof line, f)) {
        const char* q0 = strchr(line, '"');
        const char* q1 = q0 ? strchr(q0 + 1, '"') : nullptr;
        const char* body = q1 ? strstr(q1, "{\"nb\":") : nullptr;
        TuneEntry e;
        if (body && sscanf(body, "{\"nb\": %d, \"gemm\": %d, \"ms\": %lf", &e.nb, &e.gemm, &e.ms) == 3)
            m[std::string(q0 + 1, q1)] = e;
    }
    fclose(f);
    return m;
}

static bool tune_write(const char* path, const std::map<std::string, TuneEntry>& m)
{
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "w");
    if (!f) return false;
    fprintf(f, "{\n\"format\": \"binary16 grouped-LU tuning table, one entry per N bucket\",\n\"entries\": {\n");
    size_t k = 0;
    for (const auto& kv : m)
        fprintf(f, "  \"%s\": {\"nb\": %d, \"gemm\": %d, \"ms\": %.6f}%s\n", kv.first.c_str(), kv.second.nb,
                kv.second.gemm, kv.second.ms, ++k < m.size() ? "," : "");
    fprintf(f, "}\n}\n");
    const bool ok = fclose(f) == 0;
    return ok && rename(tmp.c_str(), path) == 0;
}

static bool tune_valid(int nb, int g)
{
    if (nb < 16 || nb > 128 || nb % 16 || g < 1 || g > 5) return false;
    if (g == 2) return nb % 64 == 0 && tc_gemm_supported();
    if (g == 5) return nb == 64 && tc_gemm_supported();
    if (g >= 3) return nb <= 64 && tc_gemm_supported();
    return true;
}

// Times the grouped binary16 LU of each bucket alone on the batch's initial
// Jacobians for each candidate (outer block, update / launch form) and keeps
// the fastest; a bucket found in the tuning table takes the stored choice.
static nl_status batch_autotune(nl_batch* B)
{
    const int cands[7][2] = {{128, 2}, {64, 2}, {64, 5}, {64, 3}, {64, 4}, {32, 3}, {32, 4}};
    const bool tc = tc_gemm_supported();
    const char* path = getenv("NL_LU_TUNE_FILE");
    if (path && !*path) path = nullptr;
    std::map<std::string, TuneEntry> table = tune_read(path);
    bool dirty = false;
    cudaEvent_t e0, e1;
    NL_CUDA_OK(cudaEventCreate(&e0));
    NL_CUDA_OK(cudaEventCreate(&e1));
    // F and J at x0 = ones for every instance
    k_b_init<<<B->count, 256, 0, B->st>>>(B->dinst, B->dst);
    NL_TRY(launch_residual_g(B->dinst, B->dst, B->res_tasks, B->n_res, 0, B->htab, B->st));
    nl_status s = NL_OK;
    for (int b = 0; b < B->nbk && s == NL_OK; ++b) {
        const std::string key = tune_key(B, b);
        auto it = table.find(key);
        if (it != table.end() && tune_valid(it->second.nb, it->second.gemm)) {
            B->bk_nb[b] = it->second.nb;
            B->bk_gemm[b] = it->second.gemm;
            B->bk_cached[b] = 1;
            continue;
        }
        double best = 1e300;
        int bnb = 128, bg = tc ? 2 : 1;
        for (const auto& cnd : cands) {
            const int nb = cnd[0], g = cnd[1];
            if (g >= 2 && !tc) continue;
            GroupPlan pl;
            if ((s = batch_plan16(B, b, nb, g, &pl)) != NL_OK) break;
            float ms_best = 1e30f;
            for (int rep = 0; rep < 2 && s == NL_OK; ++rep) {
                if (cudaMemsetAsync(B->flags, 0, sizeof(int) * B->count, B->st) != cudaSuccess) s = NL_ECUDA;
                if (s == NL_OK)
                    s = launch_jacobian_g(B->dinst, B->dst, B->row_off, B->count, B->total_rows, B->htab, B->htab32,
                                          0, B->st);
                if (s != NL_OK) break;
                cudaEventRecord(e0, B->st);
                s = lu_grouped_factor(pl, B->bk_gin[b], B->st, nullptr);
                cudaEventRecord(e1, B->st);
                if (s == NL_OK && cudaEventSynchronize(e1) != cudaSuccess) s = NL_ECUDA;
                float ms = 0.0f;
                if (s == NL_OK) cudaEventElapsedTime(&ms, e0, e1);
                ms_best = std::min(ms_best, ms);
            }
            lu_grouped_free(&pl);
            if (s != NL_OK) break;
            B->tune_bucket.push_back(b);
            B->tune_nb.push_back(nb);
            B->tune_gemm.push_back(g);
            B->tune_ms.push_back(ms_best);
            if (ms_best < best) {
                best = ms_best;
                bnb = nb;
                bg = g;
            }
        }
        B->bk_nb[b] = bnb;
        B->bk_gemm[b] = bg;
        table[key] = TuneEntry{bnb, bg, best};
        dirty = true;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s == NL_OK && dirty && path) tune_write(path, table);  // best effort: an unwritable table only costs tuning
    return s;
}

static nl_status batch_alloc_fp64(nl_batch* B);

extern "C" {

nl_status nl_batch_create(int count, const int64_t* N, const double* c, const nl_config* cfg, nl_batch** out)
{
    set_error("");
    if (count < 1 || !N || !c || !out) {
        set_error("nl_batch_create: need count >= 1, N, c and out");
        return NL_EINVAL;
    }
    nl_config d;
    nl_config_default(&d);
    if (cfg) d = *cfg;
    if (d.gmres_restart < 1 || d.gmres_restart > 62 || d.ir_maxit < 0 || d.newton_maxit < 0 ||
        d.newton_maxit >= NL_MAX_HIST || (d.lu_nb && (d.lu_nb < 16 || d.lu_nb > 128 || d.lu_nb % 16)) ||
        d.lu_path < 0 || d.lu_path > 1 ||
        !(d.trsv_cluster == -1 || d.trsv_cluster == 0 || d.trsv_cluster == 4 || d.trsv_cluster == 8 ||
          d.trsv_cluster == 16) ||
        !(d.lu_stream == 0 || d.lu_stream == -1 || d.lu_stream == 256) || d.ir_variant != 0 ||
        d.trailing_gemm < 0 || d.trailing_gemm > 5 ||
        d.gmres_factors32 != 0 || d.lu16_arith != 0 || d.scale_fp16 != 0) {
        set_error("nl_batch_create: invalid configuration");
        return NL_EINVAL;
    }
    for (int i = 0; i < count; ++i)
        if (N[i] < 1 || N[i] > kBMaxN || !(c[i] >= 0.0 && c[i] < 1.0)) {
            set_error("nl_batch_create: instance %d needs N in [1, %d] and 0 <= c < 1", i, kBMaxN);
            return NL_EINVAL;
        }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        set_error("nl_batch_create: no CUDA device");
        return NL_ECUDA;
    }
    nl_batch* B = new nl_batch();
    B->count = count;
    B->cfg = d;
    B->N.resize(count);
    B->c.assign(c, c + count);
    B->off.resize(count + 1, 0);
    B->ld.resize(count);
    for (int i = 0; i < count; ++i) {
        B->N[i] = (int)N[i];
        B->off[i + 1] = B->off[i] + N[i];
        B->ld[i] = (int)round_up(N[i], 64);
        B->nmax = std::max(B->nmax, B->N[i]);
    }
    B->total_rows = (int)B->off[count];
    const int64_t tot = B->off[count];
    if (cudaStreamCreateWithFlags(&B->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&B->s1, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&B->s2, cudaStreamNonBlocking) != cudaSuccess) {
        set_error("nl_batch_create: stream creation failed");
        B->own_streams = true;
        batch_free(B);
        return NL_ECUDA;
    }
    B->own_streams = true;
    tc_gemm_supported();  // one-time set-ups outside any capture
    if (batch_trsv_smem_setup() != NL_OK || lu_grouped_setup() != NL_OK) {
        batch_free(B);
        return NL_ECUDA;
    }
    // task lists (largest instances first)
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return B->N[a] > B->N[b]; });
    std::vector<BTask> rt, gt;
    for (int i : order) {
        for (int i0 = 0; i0 < B->N[i]; i0 += residual_block_rows()) rt.push_back({i, i0});
        for (int i0 = 0; i0 < B->N[i]; i0 += gemv_block_rows()) gt.push_back({i, i0});
    }
    B->n_res = (int)rt.size();
    B->n_gemv = (int)gt.size();
    std::vector<int> row_off(count + 1);
    for (int i = 0; i <= count; ++i) row_off[i] = (int)B->off[i];
    // sizes
    auto carve = [&](Carver& cv) {
        cv.take<BInst>(count);
        cv.take<GInst>(count);
        cv.take<GInst>(count);
        cv.take<GInst>(count);  // bucket tables
        cv.take<BState>(count);
        cv.take<BCtl>(1);
        cv.take<BParams>(1);
        cv.take<int>(count);  // flags
        cv.take<BTask>(rt.size());
        cv.take<BTask>(gt.size());
        cv.take<int>(count + 1);
        cv.take<int>(count);
        cv.take<double>(2 * (size_t)B->nmax);
        cv.take<float>(2 * (size_t)B->nmax);
        cv.take<double>(tot);  // x0
        cv.take<double>(tot);  // xout
        cv.take<double>((size_t)count * NL_MAX_HIST);
        cv.take<int>((size_t)count * NL_MAX_HIST * 3);
        cv.take<double>((size_t)count * NL_MAX_HIST);
        for (int i = 0; i < count; ++i) {
            const int n = B->N[i];
            const size_t ld = B->ld[i];
            for (int q = 0; q < 4; ++q) cv.take<double>(n);  // x[0], x[1], F, rr
            cv.take<float>((size_t)n * ld);                  // J32
            cv.take<__half>((size_t)n * ld);                 // J16
            cv.take<int>(n);                                 // ipiv
            for (int q = 0; q < 3; ++q) cv.take<float>(ld);  // b u r
            cv.take<double>(cdiv(n, gemv_block_rows()) + 64);
            cv.take<unsigned>(16);
            cv.take<char>(lu_stage_bytes());
            cv.take<__half>((size_t)round_up(n, 128) * 128);  // U12^T
        }
    };
    {
        Carver cv(nullptr);
        carve(cv);
        B->pool_bytes = cv.off + 256;
    }
    if (dev_malloc(&B->pool, B->pool_bytes) != cudaSuccess) {
        cudaGetLastError();
        set_error("nl_batch_create: cudaMalloc of %zu bytes failed", B->pool_bytes);
        batch_free(B);
        return NL_ENOMEM;
    }
    cudaMemset(B->pool, 0, B->pool_bytes);
    Carver cv(B->pool);
    B->dinst = cv.take<BInst>(count);
    B->gin = cv.take<GInst>(count);
    B->gin64 = cv.take<GInst>(count);
    GInst* bk_base = cv.take<GInst>(count);
    B->dst = cv.take<BState>(count);
    B->ctl = cv.take<BCtl>(1);
    B->prm = cv.take<BParams>(1);
    int* flags = cv.take<int>(count);
    B->flags = flags;
    B->res_tasks = cv.take<BTask>(rt.size());
    B->gemv_tasks = cv.take<BTask>(gt.size());
    B->row_off = cv.take<int>(count + 1);
    B->order = cv.take<int>(count);
    B->htab = cv.take<double>(2 * (size_t)B->nmax);
    B->htab32 = cv.take<float>(2 * (size_t)B->nmax);
    B->x0 = cv.take<double>(tot);
    B->xout = cv.take<double>(tot);
    B->hist = cv.take<double>((size_t)count * NL_MAX_HIST);
    B->lin_iters = cv.take<int>((size_t)count * NL_MAX_HIST * 3);
    B->lin_outer = B->lin_iters + (size_t)count * NL_MAX_HIST;
    B->lin_failed = B->lin_outer + (size_t)count * NL_MAX_HIST;
    B->lin_relres = cv.take<double>((size_t)count * NL_MAX_HIST);
    B->hinst.resize(count);
    B->hgin.resize(count);
    for (int i = 0; i < count; ++i) {
        const int n = B->N[i];
        const size_t ld = B->ld[i];
        BInst& I = B->hinst[i];
        memset(&I, 0, sizeof(I));
        I.N = n;
        I.ld = (int)ld;
        I.c = B->c[i];
        I.x[0] = cv.take<double>(n);
        I.x[1] = cv.take<double>(n);
        I.F = cv.take<double>(n);
        I.rr = cv.take<double>(n);
        I.J32 = cv.take<float>((size_t)n * ld);
        __half* J16 = cv.take<__half>((size_t)n * ld);
        I.J = J16;
        I.ipiv = cv.take<int>(n);
        I.flag = flags + i;
        I.b = cv.take<float>(ld);
        I.u = cv.take<float>(ld);
        I.r = cv.take<float>(ld);
        I.part = cv.take<double>(cdiv(n, gemv_block_rows()) + 64);
        I.cnt = cv.take<unsigned>(16);
        void* stage = cv.take<char>(lu_stage_bytes());
        __half* ut = cv.take<__half>((size_t)round_up(n, 128) * 128);
        I.x0 = B->x0 + B->off[i];
        I.xout = B->xout + B->off[i];
        GInst& G = B->hgin[i];
        G.A = J16;
        G.ld = (int64_t)ld;
        G.N = n;
        G.pad = 0;
        G.ipiv = I.ipiv;
        G.flag = I.flag;
        G.stage = stage;
        G.ut = ut;
    }
    // N buckets: bucket tables in instance order, one stream and event each
    {
        int cnt[kBMaxBuckets] = {}, idx[kBMaxBuckets];
        std::vector<int> raw(count);
        for (int i = 0; i < count; ++i) {
            int b = 0;
            while (B->N[i] > kBucketNmax[b]) ++b;
            raw[i] = b;
            cnt[b] += 1;
        }
        B->nbk = 0;
        for (int b = 0; b < kBMaxBuckets; ++b) {
            idx[b] = -1;
            if (!cnt[b]) continue;
            idx[b] = B->nbk;
            B->bk_id[B->nbk] = b;
            B->bk_nmax[B->nbk] = kBucketNmax[b];
            B->bk_count[B->nbk] = cnt[b];
            B->nbk += 1;
        }
        B->bk_of.resize(count);
        B->bk_hgin.assign(B->nbk, {});
        for (int i = 0; i < count; ++i) {
            B->bk_of[i] = idx[raw[i]];
            B->bk_hgin[B->bk_of[i]].push_back(B->hgin[i]);
        }
        size_t o = 0;
        for (int b = 0; b < B->nbk; ++b) {
            B->bk_gin[b] = bk_base + o;
            if (cudaMemcpy(B->bk_gin[b], B->bk_hgin[b].data(), sizeof(GInst) * B->bk_count[b],
                           cudaMemcpyHostToDevice) != cudaSuccess) {
                set_error("nl_batch_create: table upload failed");
                batch_free(B);
                return NL_ECUDA;
            }
            o += B->bk_count[b];
        }
        if (B->nbk > 1) {
            bool ok = cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming) == cudaSuccess;
            for (int b = 0; b < B->nbk && ok; ++b)
                ok = cudaStreamCreateWithFlags(&B->bk_st[b], cudaStreamNonBlocking) == cudaSuccess &&
                     cudaEventCreateWithFlags(&B->bk_ev[b], cudaEventDisableTiming) == cudaSuccess;
            if (!ok) {
                set_error("nl_batch_create: stream creation failed");
                batch_free(B);
                return NL_ECUDA;
            }
        }
    }
    if (cudaMemcpy(B->dinst, B->hinst.data(), sizeof(BInst) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(B->gin, B->hgin.data(), sizeof(GInst) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(B->res_tasks, rt.data(), sizeof(BTask) * rt.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(B->gemv_tasks, gt.data(), sizeof(BTask) * gt.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(B->row_off, row_off.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(B->order, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice) != cudaSuccess) {
        set_error("nl_batch_create: table upload failed");
        batch_free(B);
        return NL_ECUDA;
    }
    k_htab_g<<<(unsigned)cdiv(2 * (int64_t)B->nmax, 256), 256, 0, B->st>>>(2 * B->nmax - 1, B->htab, B->htab32);
    // x0 = ones for the autotuner's Jacobians
    {
        std::vector<double> ones((size_t)tot, 1.0);
        if (cudaMemcpy(B->x0, ones.data(), sizeof(double) * tot, cudaMemcpyHostToDevice) != cudaSuccess) {
            set_error("nl_batch_create: upload failed");
            batch_free(B);
            return NL_ECUDA;
        }
    }
    nl_status s = NL_OK;
    if (d.lu_nb) {
        int g = d.trailing_gemm ? d.trailing_gemm : 2;
        if (g == 2 && (d.lu_nb % 64 || !tc_gemm_supported())) g = 1;
        if (g >= 3 && (d.lu_nb > 64 || !tc_gemm_supported())) g = 1;
        if (g == 5 && d.lu_nb != 64) g = 1;
        for (int b = 0; b < B->nbk; ++b) {
            B->bk_nb[b] = d.lu_nb;
            B->bk_gemm[b] = g;
        }
    } else {
        s = batch_autotune(B);
    }
    for (int b = 0; b < B->nbk && s == NL_OK; ++b) s = batch_plan16(B, b, B->bk_nb[b], B->bk_gemm[b], &B->bk_plan[b]);
    B->nb = B->bk_nb[B->nbk - 1];
    B->gemm = B->bk_gemm[B->nbk - 1];
    double lu16_ms = 0.0;
    if (s == NL_OK) s = batch_time_lu16(B, &lu16_ms);
    if (s == NL_OK && cudaStreamSynchronize(B->st) != cudaSuccess) {
        set_error("nl_batch_create: %s", cudaGetErrorString(cudaGetLastError()));
        s = NL_ECUDA;
    }
    if (s != NL_OK) {
        batch_free(B);
        return s;
    }
    B->stats.resize(count);
    memset(&B->info, 0, sizeof(B->info));
    B->info.tune_count = (int)std::min<size_t>(NL_BATCH_MAX_TUNE, B->tune_nb.size());
    for (int k = 0; k < B->info.tune_count; ++k) {
        B->info.tune_bucket[k] = B->tune_bucket[k];
        B->info.tune_nb[k] = B->tune_nb[k];
        B->info.tune_gemm[k] = B->tune_gemm[k];
        B->info.tune_ms[k] = B->tune_ms[k];
    }
    B->info.lu16_ms = lu16_ms;
    B->info.nbuckets = B->nbk;
    for (int b = 0; b < B->nbk; ++b) {
        B->info.bucket_nmax[b] = B->bk_nmax[b];
        B->info.bucket_count[b] = B->bk_count[b];
        B->info.bucket_nb[b] = B->bk_nb[b];
        B->info.bucket_gemm[b] = B->bk_gemm[b];
        B->info.bucket_cached[b] = B->bk_cached[b];
    }
    B->info.lu_nb = B->nb;
    B->info.trailing_gemm = B->gemm;
    *out = B;
    return NL_OK;
}

}  // extern "C"

static nl_status batch_alloc_fp64(nl_batch* B)
{
    if (B->pool64) return NL_OK;
    const int count = B->count;
    size_t bytes;
    {
        Carver cv(nullptr);
        cv.take<BInst>(count);
        for (int i = 0; i < count; ++i) {
            cv.take<double>((size_t)B->N[i] * B->ld[i]);
            cv.take<double>(B->ld[i]);
            cv.take<double>(B->ld[i]);
        }
        bytes = cv.off + 256;
    }
    if (dev_malloc(&B->pool64, bytes) != cudaSuccess) {
        cudaGetLastError();
        B->pool64 = nullptr;
        set_error("batch: cudaMalloc of %zu bytes for the double Jacobians failed", bytes);
        return NL_ENOMEM;
    }
    B->pool64_bytes = bytes;
    NL_CUDA_OK(cudaMemset(B->pool64, 0, bytes));
    Carver cv(B->pool64);
    B->dinst64 = cv.take<BInst>(count);
    B->hinst64 = B->hinst;
    B->hgin64 = B->hgin;
    for (int i = 0; i < count; ++i) {
        double* J64 = cv.take<double>((size_t)B->N[i] * B->ld[i]);
        B->hinst64[i].J = J64;
        B->hinst64[i].b64 = cv.take<double>(B->ld[i]);
        B->hinst64[i].u64 = cv.take<double>(B->ld[i]);
        B->hgin64[i].A = J64;
        B->hgin64[i].ut = nullptr;
    }
    NL_CUDA_OK(cudaMemcpy(B->dinst64, B->hinst64.data(), sizeof(BInst) * count, cudaMemcpyHostToDevice));
    NL_CUDA_OK(cudaMemcpy(B->gin64, B->hgin64.data(), sizeof(GInst) * count, cudaMemcpyHostToDevice));
    return lu_grouped_plan(count, B->hgin64.data(), 64, 1, true, &B->plan64);
}

// Captures the whole batched solve of one mode (0 three precisions, 1 FP64)
// into a graph with WHILE nodes for the Newton steps and the IR corrections.
static nl_status batch_build_graph(nl_batch* B, int fp64)
{
    const int count = B->count;
    const nl_config& C = B->cfg;
    const BInst* inst = fp64 ? B->dinst64 : B->dinst;
    const GInst* gin64 = B->gin64;
    BParams* prm = B->prm;
    cudaStream_t s0 = B->st, s1 = B->s1, s2 = B->s2;
    const size_t vec_smem = (size_t)round_up(B->nmax, 32) * (fp64 ? 8 : 4);
    int nodes_step = 0, nodes_ir = 0;
    NL_CUDA_OK(cudaStreamBeginCapture(s0, cudaStreamCaptureModeRelaxed));
    nl_status s = NL_OK;
    cudaGraph_t g = nullptr;
    do {
        if (cudaMemsetAsync(B->ctl, 0, sizeof(BCtl), s0) != cudaSuccess) { s = NL_ECUDA; break; }
        k_b_init<<<count, 256, 0, s0>>>(inst, B->dst);
        if ((s = launch_residual_g(inst, B->dst, B->res_tasks, B->n_res, 0, B->htab, s0)) != NL_OK) break;
        // tol and tau_a come from device memory so that one graph serves every tolerance
        k_b_init_check<<<1, 256, 0, s0>>>(inst, B->dst, count, prm, C.newton_maxit, B->hist, B->ctl);
        cudaGraphConditionalHandle hN, hI;
        {
            cudaStreamCaptureStatus cs;
            cudaGraph_t cg;
            if (cudaStreamGetCaptureInfo(s0, &cs, nullptr, &cg, nullptr, nullptr, nullptr) != cudaSuccess ||
                cudaGraphConditionalHandleCreate(&hN, cg, 0, cudaGraphCondAssignDefault) != cudaSuccess) {
                s = NL_ECUDA;
                break;
            }
        }
        k_b_cond<<<1, 1, 0, s0>>>(B->ctl, 0, 1, C.newton_maxit, hN);
        if ((s = add_while_node(s0, s1, hN)) != NL_OK) break;
        // ---- Newton step body (s1)
        if ((s = launch_jacobian_g(inst, B->dst, B->row_off, count, B->total_rows, B->htab, B->htab32, fp64, s1)) !=
            NL_OK)
            break;
        nodes_step = 1;
        // lu_path = 1 (interchanging path only): the batch factors nothing itself and hands
        // every instance to the single-instance path at its first step
        const int park_all = (C.lu_path == 1) ? 1 : 0;
        if (!park_all) {
            s = fp64 ? lu_grouped_factor(B->plan64, gin64, s1, &nodes_step) : batch_lu16(B, s1, &nodes_step);
            if (s != NL_OK) break;
        }
        if (!fp64) {
            k_b_rhs<<<count, 256, 0, s1>>>(inst, B->dst, C.eta_j, C.ir_maxit, park_all, B->ctl);
            {
                cudaStreamCaptureStatus cs;
                cudaGraph_t cg;
                if (cudaStreamGetCaptureInfo(s1, &cs, nullptr, &cg, nullptr, nullptr, nullptr) != cudaSuccess ||
                    cudaGraphConditionalHandleCreate(&hI, cg, 0, cudaGraphCondAssignDefault) != cudaSuccess) {
                    s = NL_ECUDA;
                    break;
                }
            }
            k_b_cond<<<1, 1, 0, s1>>>(B->ctl, 1, 1, C.ir_maxit, hI);
            if ((s = add_while_node(s1, s2, hI)) != NL_OK) break;
            // ---- IR correction body (s2)
            k_b_trsv<__half, float><<<count, kBtThreads, vec_smem, s2>>>(inst, B->dst, B->order);
            if ((s = launch_gemv_residual_g(inst, B->dst, B->gemv_tasks, B->n_gemv, s2)) != NL_OK) break;
            k_b_ir_check<<<(unsigned)cdiv(count, 256), 256, 0, s2>>>(B->dst, count, C.eta_j, C.ir_maxit, B->ctl);
            k_b_cond<<<1, 1, 0, s2>>>(B->ctl, 1, 0, C.ir_maxit, hI);
            nodes_ir = 4;
            cudaGraph_t body = nullptr;
            if (cudaStreamEndCapture(s2, &body) != cudaSuccess) { s = NL_ECUDA; break; }
            if ((s = launch_residual_g(inst, B->dst, B->res_tasks, B->n_res, 1, B->htab, s1)) != NL_OK) break;
            nodes_step += 3;
        } else {
            k_b_rhs64<<<count, 256, 0, s1>>>(inst, B->dst, park_all);
            k_b_trsv<double, double><<<count, kBtThreads, vec_smem, s1>>>(inst, B->dst, B->order);
            if ((s = launch_residual_g(inst, B->dst, B->res_tasks, B->n_res, 2, B->htab, s1)) != NL_OK) break;
            nodes_step += 3;
        }
        k_b_newton_check<<<1, 256, 0, s1>>>(inst, B->dst, count, C.newton_maxit, fp64, B->hist, B->lin_iters,
                                            B->lin_outer, B->lin_failed, B->lin_relres, B->ctl);
        k_b_cond<<<1, 1, 0, s1>>>(B->ctl, 0, 0, C.newton_maxit, hN);
        nodes_step += 2;
        {
            cudaGraph_t body = nullptr;
            if (cudaStreamEndCapture(s1, &body) != cudaSuccess) { s = NL_ECUDA; break; }
        }
        k_b_gather<<<count, 256, 0, s0>>>(inst, B->dst);
    } while (0);
    if (s != NL_OK) {
        // end every capture that is still open before reporting
        cudaGraph_t junk;
        cudaStreamCaptureStatus cs;
        for (cudaStream_t q : {s2, s1, s0})
            if (cudaStreamIsCapturing(q, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
                if (cudaStreamEndCapture(q, &junk) == cudaSuccess && junk) cudaGraphDestroy(junk);
            }
        cudaGetLastError();
        if (!get_error()[0]) set_error("batch: graph capture failed");
        return s;
    }
    NL_CUDA_OK(cudaStreamEndCapture(s0, &g));
    cudaGraphExec_t ex = nullptr;
    cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        set_error("batch: graph instantiation failed: %s", cudaGetErrorString(e));
        return NL_ECUDA;
    }
    B->exec[fp64] = ex;
    B->nodes_newton[fp64] = nodes_step;
    B->nodes_ir = nodes_ir;
    B->nodes_init = 5;
    return NL_OK;
}

static nl_status status_of(int bs)
{
    switch (bs) {
    case BS_CONVERGED: return NL_OK;
    case BS_NOTCONV: return NL_ENOTCONV;
    case BS_NUMERIC: return NL_ENUMERIC;
    default: return NL_ENOTCONV;
    }
}

static nl_status batch_solve_impl(nl_batch* B, const double* x0, bool x0_host, double tol, nl_mode mode,
                                  double* x_out, bool out_host)
{
    auto t0 = std::chrono::steady_clock::now();
    const int count = B->count;
    const int fp64 = (mode == NL_FP64LU) ? 1 : 0;
    if (fp64) NL_TRY(batch_alloc_fp64(B));
    if (!B->exec[fp64]) NL_TRY(batch_build_graph(B, fp64));
    cudaStream_t st = B->st;
    const int64_t tot = B->off[count];
    if (x0) {
        NL_CUDA_OK(cudaMemcpyAsync(B->x0, x0, sizeof(double) * tot,
                                   x0_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
    } else {
        k_b_fill<<<(unsigned)cdiv(tot, 256), 256, 0, st>>>(tot, 1.0, B->x0);
    }
    BParams p{tol, B->cfg.tau_a};
    NL_CUDA_OK(cudaMemcpyAsync(B->prm, &p, sizeof(p), cudaMemcpyHostToDevice, st));
    cudaEvent_t e0, e1;
    NL_CUDA_OK(cudaEventCreate(&e0));
    NL_CUDA_OK(cudaEventCreate(&e1));
    cudaEventRecord(e0, st);
    cudaError_t le = cudaGraphLaunch(B->exec[fp64], st);
    cudaEventRecord(e1, st);
    if (le != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        set_error("batch: graph launch failed: %s", cudaGetErrorString(le));
        return NL_ECUDA;
    }
    std::vector<BState> hs(count);
    BCtl ctl;
    NL_CUDA_OK(cudaMemcpyAsync(hs.data(), B->dst, sizeof(BState) * count, cudaMemcpyDeviceToHost, st));
    NL_CUDA_OK(cudaMemcpyAsync(&ctl, B->ctl, sizeof(BCtl), cudaMemcpyDeviceToHost, st));
    NL_CUDA_OK(cudaStreamSynchronize(st));
    float gms = 0.0f;
    cudaEventElapsedTime(&gms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    {
        unsigned* tce = tc_error_word();
        unsigned e = 0;
        if (tce) NL_CUDA_OK(cudaMemcpy(&e, tce, sizeof(unsigned), cudaMemcpyDeviceToHost));
        if (e) {
            cudaMemset(tce, 0, sizeof(unsigned));
            set_error("batch: a bounded device wait of the grouped LU gave up");
            return NL_ETIMEOUT;
        }
    }
    nl_batch_info_t& In = B->info;
    const int tune_count = In.tune_count;
    In.count = count;
    In.converged = In.parked_lu = In.parked_ir = 0;
    In.newton_rounds = ctl.newton_round;
    In.ir_rounds = ctl.ir_total;
    In.lu_nb = fp64 ? 64 : B->nb;
    In.trailing_gemm = fp64 ? 1 : B->gemm;
    In.graph_nodes_step = B->nodes_newton[fp64];
    In.graph_nodes_ir = fp64 ? 0 : B->nodes_ir;
    In.gpu_launches = B->nodes_init + ctl.newton_round * B->nodes_newton[fp64] + (fp64 ? 0 : ctl.ir_total * B->nodes_ir);
    In.t_graph_ms = gms;
    In.tune_count = tune_count;
    B->stats_ready = false;
    B->last_fp64 = fp64;
    B->single.assign(count, nl_stats_t());
    B->single_used.assign(count, 0);
    B->hstate = hs;
    // instances that left the batch: finish them one by one
    auto ts = std::chrono::steady_clock::now();
    nl_status result = NL_OK;
    for (int i = 0; i < count; ++i) {
        const BState& S = hs[i];
        if (S.status == BS_PARKED_LU || S.status == BS_PARKED_IR) {
            (S.status == BS_PARKED_LU ? In.parked_lu : In.parked_ir) += 1;
            nl_config cf = B->cfg;
            cf.tau_a = S.tau;
            if (!fp64) {
                // the same factorisation (rounding period) as the instance's bucket; the persistent
                // launch's arithmetic is the SIMT update's
                const int b = B->bk_of[i];
                cf.lu_nb = B->bk_nb[b];
                cf.trailing_gemm = B->bk_gemm[b] == 5 ? 2 : (B->bk_gemm[b] >= 3 ? 1 : B->bk_gemm[b]);
            }
            cf.newton_maxit = std::max(0, B->cfg.newton_maxit - S.it);
            nl_solver* sv = nullptr;
            nl_status cs = nl_create(B->N[i], B->c[i], &cf, &sv);
            if (cs != NL_OK) return cs;
            nl_set_stream(sv, st);
            const nl_mode m = fp64 ? NL_FP64LU : (S.status == BS_PARKED_IR ? NL_GMRESIR16 : NL_IR16_GMRES);
            const double* xcur = B->hinst[i].x[S.par];
            cs = nl_solve_device(sv, xcur, 0.0, m, B->hinst[i].xout);
            nl_stats(sv, &B->single[i]);
            B->single_used[i] = 1;
            In.gpu_launches += B->single[i].gpu_launches;
            nl_destroy(sv);
            if (cs != NL_OK && cs != NL_ENOTCONV && cs != NL_ENUMERIC && cs != NL_ESINGULAR) return cs;
            if (cs == NL_OK) In.converged += 1;
            else if (result == NL_OK) result = cs;
        } else if (S.status == BS_CONVERGED) {
            In.converged += 1;
        } else if (result == NL_OK) {
            result = status_of(S.status);
        }
    }
    In.t_single_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - ts).count();
    NL_CUDA_OK(cudaMemcpyAsync(x_out, B->xout, sizeof(double) * tot,
                               out_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    NL_CUDA_OK(cudaStreamSynchronize(st));
    In.t_total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return result;
}

static nl_status batch_fetch_stats(nl_batch* B)
{
    if (B->stats_ready) return NL_OK;
    const size_t n = (size_t)B->count * NL_MAX_HIST;
    std::vector<double> hist(n), rel(n);
    std::vector<int> li(3 * n);
    NL_CUDA_OK(cudaMemcpy(hist.data(), B->hist, sizeof(double) * n, cudaMemcpyDeviceToHost));
    NL_CUDA_OK(cudaMemcpy(rel.data(), B->lin_relres, sizeof(double) * n, cudaMemcpyDeviceToHost));
    NL_CUDA_OK(cudaMemcpy(li.data(), B->lin_iters, sizeof(int) * 3 * n, cudaMemcpyDeviceToHost));
    for (int i = 0; i < B->count; ++i) {
        const BState& S = B->hstate[i];
        nl_stats_t& o = B->stats[i];
        memset(&o, 0, sizeof(o));
        o.mode = B->last_fp64 ? NL_FP64LU : NL_IR16_GMRES;
        o.lu_nb = B->last_fp64 ? 64 : B->bk_nb[B->bk_of[i]];
        o.fnorm0 = S.fn0;
        o.fnorm = S.fn;
        o.status = status_of(S.status);
        int it = S.it;
        for (int k = 0; k <= it && k < NL_MAX_HIST; ++k) o.hist[k] = hist[(size_t)i * NL_MAX_HIST + k];
        for (int k = 0; k < it && k < NL_MAX_HIST; ++k) {
            o.lin_iters[k] = li[(size_t)i * NL_MAX_HIST + k];
            o.lin_outer[k] = li[n + (size_t)i * NL_MAX_HIST + k];
            o.lin_failed[k] = li[2 * n + (size_t)i * NL_MAX_HIST + k];
            o.lin_relres[k] = rel[(size_t)i * NL_MAX_HIST + k];
        }
        if (B->single_used[i]) {
            const nl_stats_t& s1 = B->single[i];
            const double scale = (S.fn0 > 0.0) ? s1.fnorm0 / S.fn0 : 0.0;
            for (int k = 0; k < s1.newton_iters && it + k < NL_MAX_HIST - 1; ++k) {
                o.hist[it + k + 1] = s1.hist[k + 1] * scale;
                o.lin_iters[it + k] = s1.lin_iters[k];
                o.lin_outer[it + k] = s1.lin_outer[k];
                o.lin_failed[it + k] = s1.lin_failed[k];
                o.lin_relres[it + k] = s1.lin_relres[k];
            }
            if (S.status == BS_PARKED_IR && s1.newton_iters > 0) {
                // the stalled IR attempt belongs to the step GMRES-IR redid
                o.lin_iters[it] += S.lin_iters;
                o.lin_outer[it] += S.outer;
                o.lin_failed[it] = 1;
            }
            it += s1.newton_iters;
            o.status = s1.status;
            o.fnorm = s1.fnorm;
            o.lu_pivoted = s1.lu_pivoted;
        }
        o.newton_iters = it;
    }
    B->stats_ready = true;
    return NL_OK;
}

extern "C" {

nl_status nl_batch_solve(nl_batch* b, const double* x0, double tol, nl_mode mode, double* x_out)
{
    set_error("");
    if (!b || !x_out || !(mode == NL_FP64LU || mode == NL_IR16_GMRES) || !(tol >= 0.0)) {
        set_error("nl_batch_solve: bad argument (modes: NL_IR16_GMRES, NL_FP64LU)");
        return NL_EINVAL;
    }
    return batch_solve_impl(b, x0, true, tol, mode, x_out, true);
}

nl_status nl_batch_solve_device(nl_batch* b, const double* x0_dev, double tol, nl_mode mode, double* x_out_dev)
{
    set_error("");
    if (!b || !x_out_dev || !(mode == NL_FP64LU || mode == NL_IR16_GMRES) || !(tol >= 0.0)) {
        set_error("nl_batch_solve_device: bad argument (modes: NL_IR16_GMRES, NL_FP64LU)");
        return NL_EINVAL;
    }
    return batch_solve_impl(b, x0_dev, false, tol, mode, x_out_dev, false);
}

nl_status nl_batch_stats(nl_batch* b, int i, nl_stats_t* out)
{
    if (!b || !out || i < 0 || i >= b->count || b->hstate.empty()) {
        set_error("nl_batch_stats: bad argument or no solve yet");
        return NL_EINVAL;
    }
    NL_TRY(batch_fetch_stats(b));
    *out = b->stats[i];
    return NL_OK;
}

nl_status nl_batch_info(const nl_batch* b, nl_batch_info_t* out)
{
    if (!b || !out) {
        set_error("nl_batch_info: NULL argument");
        return NL_EINVAL;
    }
    *out = b->info;
    return NL_OK;
}

nl_status nl_batch_set_stream(nl_batch* b, void* stream)
{
    if (!b) {
        set_error("nl_batch_set_stream: NULL handle");
        return NL_EINVAL;
    }
    if (b->own_st && b->st) {
        cudaStreamSynchronize(b->st);
        cudaStreamDestroy(b->st);
    }
    b->own_st = false;
    b->st = (cudaStream_t)stream;
    return NL_OK;
}

int64_t nl_batch_device_bytes(const nl_batch* b) { return b ? (int64_t)(b->pool_bytes + b->pool64_bytes) : 0; }

void nl_batch_destroy(nl_batch* b) { batch_free(b); }

nl_status nl_lu_grouped(int count, const int64_t* N, void* const* A, const int64_t* ld, int32_t* const* ipiv,
                        int fp64, int nb, int gemm, int32_t* flags_host, void* stream)
{
    set_error("");
    if (count < 1 || !N || !A || !ld || !ipiv || !flags_host || gemm < 0 || gemm > 5) {
        set_error("nl_lu_grouped: bad argument");
        return NL_EINVAL;
    }
    for (int i = 0; i < count; ++i)
        if (N[i] < 1 || N[i] > 32768 || ld[i] < N[i] || ld[i] % 8 || !A[i] || !ipiv[i]) {
            set_error("nl_lu_grouped: matrix %d: need N in [1, 32768], ld >= N, ld a multiple of 8", i);
            return NL_EINVAL;
        }
    if (nb == 0) nb = fp64 ? 64 : 128;
    if (gemm == 0) gemm = 2;
    cudaStream_t st = (cudaStream_t)stream;
    size_t bytes = 0;
    {
        Carver cv(nullptr);
        cv.take<GInst>(count);
        cv.take<int>(count);
        for (int i = 0; i < count; ++i) {
            cv.take<char>(lu_stage_bytes());
            cv.take<__half>((size_t)round_up(N[i], 128) * 128);
        }
        bytes = cv.off + 256;
    }
    void* wk = nullptr;
    NL_CUDA_OK(cudaMalloc(&wk, bytes));
    Carver cv(wk);
    GInst* dg = cv.take<GInst>(count);
    int* flags = cv.take<int>(count);
    std::vector<GInst> hg(count);
    for (int i = 0; i < count; ++i) {
        hg[i].A = A[i];
        hg[i].ld = ld[i];
        hg[i].N = (int)N[i];
        hg[i].pad = 0;
        hg[i].ipiv = ipiv[i];
        hg[i].flag = flags + i;
        hg[i].stage = cv.take<char>(lu_stage_bytes());
        hg[i].ut = fp64 ? nullptr : cv.take<__half>((size_t)round_up(N[i], 128) * 128);
    }
    GroupPlan plan;
    nl_status s = NL_OK;
    if (cudaMemcpy(dg, hg.data(), sizeof(GInst) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(flags, 0, sizeof(int) * count) != cudaSuccess) {
        set_error("nl_lu_grouped: upload failed");
        s = NL_ECUDA;
    }
    if (s == NL_OK) {
        if (gemm == 5) s = lu_grouped_plan(count, hg.data(), nb, 2, fp64 != 0, &plan, 1, 128);
        else if (gemm >= 3) s = lu_grouped_plan(count, hg.data(), nb, 1, fp64 != 0, &plan, 1, gemm == 3 ? 64 : 128);
        else s = lu_grouped_plan(count, hg.data(), nb, gemm, fp64 != 0, &plan);
    }
    if (s == NL_OK) s = lu_grouped_factor(plan, dg, st, nullptr);
    if (s == NL_OK && cudaStreamSynchronize(st) != cudaSuccess) {
        set_error("nl_lu_grouped: %s", cudaGetErrorString(cudaGetLastError()));
        s = NL_ECUDA;
    }
    std::vector<int> hf(count, 0);
    if (s == NL_OK && cudaMemcpy(hf.data(), flags, sizeof(int) * count, cudaMemcpyDeviceToHost) != cudaSuccess)
        s = NL_ECUDA;
    lu_grouped_free(&plan);
    cudaFree(wk);
    if (s == NL_OK) {
        unsigned* tce = tc_error_word();
        unsigned e = 0;
        if (tce && cudaMemcpy(&e, tce, sizeof(unsigned), cudaMemcpyDeviceToHost) == cudaSuccess && e) {
            cudaMemset(tce, 0, sizeof(unsigned));
            set_error("nl_lu_grouped: a bounded device wait gave up");
            return NL_ETIMEOUT;
        }
        for (int i = 0; i < count; ++i) flags_host[i] = hf[i] & 1;
    }
    return s;
}

nl_status nl_lusolve_grouped(int count, const int64_t* N, const void* const* LU, const int64_t* ld,
                             const int32_t* const* ipiv, void* const* b, int fp64, void* stream)
{
    set_error("");
    if (count < 1 || !N || !LU || !ld || !ipiv || !b) {
        set_error("nl_lusolve_grouped: bad argument");
        return NL_EINVAL;
    }
    int nmax = 0;
    std::vector<GSolve> items(count);
    for (int i = 0; i < count; ++i) {
        if (N[i] < 1 || N[i] > kBMaxN || ld[i] < N[i] || !LU[i] || !ipiv[i] || !b[i]) {
            set_error("nl_lusolve_grouped: system %d: need N in [1, %d], ld >= N", i, kBMaxN);
            return NL_EINVAL;
        }
        items[i] = GSolve{LU[i], ld[i], (int)N[i], 0, ipiv[i], b[i]};
        nmax = std::max(nmax, (int)N[i]);
    }
    NL_TRY(batch_trsv_smem_setup());
    cudaStream_t st = (cudaStream_t)stream;
    GSolve* d = nullptr;
    NL_CUDA_OK(cudaMallocAsync((void**)&d, sizeof(GSolve) * count, st));
    NL_CUDA_OK(cudaMemcpyAsync(d, items.data(), sizeof(GSolve) * count, cudaMemcpyHostToDevice, st));
    const size_t smem = (size_t)round_up(nmax, 32) * (fp64 ? 8 : 4);
    if (fp64) k_trsv_grouped<double, double><<<count, kBtThreads, smem, st>>>(d);
    else k_trsv_grouped<__half, float><<<count, kBtThreads, smem, st>>>(d);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(d, st);
    if (e != cudaSuccess) {
        set_error("nl_lusolve_grouped: %s", cudaGetErrorString(e));
        return NL_ECUDA;
    }
    NL_CUDA_OK(cudaStreamSynchronize(st));
    return NL_OK;
}

}  // extern "C"
