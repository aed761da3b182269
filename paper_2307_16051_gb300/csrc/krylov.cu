// krylov.cu — single-precision pieces of IR and GMRES-IR (Section 2.2):
// the residual r = b - J32 u (Algorithm IR), vector norms, the scaled
// right-hand side of eq. (2.17), and modified Gram-Schmidt Arnoldi with
// Givens rotations for left-preconditioned GMRES.
//
// All reductions run in a fixed order (per-thread sequential sums, then a
// fixed shuffle tree, then per-block partials summed in block order by the
// last block), so every result is bitwise reproducible from run to run.
#include "common.cuh"
#include "internal.h"

namespace nl {

constexpr int kGemvWarps = 8;

// r_i = b_i - sum_j A_ij u_j (b NULL: r = A u).  One warp per row, float4
// loads along the row.  The dot product is accumulated in two-float
// (compensated) arithmetic: each product is split exactly with an FMA
// (a*u = p + e) and summed with error-free two-sums, so the row sum carries
// about twice the single-precision significand before the single result
// r_i is rounded once, matching an accumulation in double for the residual
// of IR (Algorithm IR) at single-precision bandwidth.  Also ||r||_2
// (double) via per-block partials.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void df_add_prod(DF& acc, float a, float x)
{
    float p = __fmul_rn(a, x);
    float pe = __fmaf_rn(a, x, -p);  // exact: a*x = p + pe
    float s, e;
    two_sum(acc.hi, p, s, e);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(e, pe));
}

__device__ __forceinline__ DF df_add(DF a, DF b)
{
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    DF r;
    r.hi = s;
    r.lo = __fadd_rn(__fadd_rn(a.lo, b.lo), e);
    return r;
}

// Row i of r = b - A u by one warp; returns r_i^2 in lane 0 (0 elsewhere).
__device__ __forceinline__ double gemv_row(int N, const float* __restrict__ A, int64_t ld,
                                           const float* __restrict__ b, const float* __restrict__ u,
                                           float* __restrict__ r, int i, int lane)
{
    double sq = 0.0;
    {
        const float* Ai = A + (int64_t)i * ld;
        const int n4 = N >> 2;
        const float4* A4 = reinterpret_cast<const float4*>(Ai);
        const float4* u4 = reinterpret_cast<const float4*>(u);
        DF s = {0.0f, 0.0f};
        int k = lane;
        // four iterations' loads in flight before their products (the same order of terms): at
        // N = 4096 a warp per row has 32 iterations, too few warps to hide the latency one at a time
        for (; k + 96 < n4; k += 128) {
            float4 a[4], x[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = __ldcs(A4 + k + 32 * q);
                x[q] = __ldg(u4 + k + 32 * q);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                df_add_prod(s, a[q].x, x[q].x);
                df_add_prod(s, a[q].y, x[q].y);
                df_add_prod(s, a[q].z, x[q].z);
                df_add_prod(s, a[q].w, x[q].w);
            }
        }
        for (; k < n4; k += 32) {
            float4 a = __ldcs(A4 + k);
            float4 x = __ldg(u4 + k);
            df_add_prod(s, a.x, x.x);
            df_add_prod(s, a.y, x.y);
            df_add_prod(s, a.z, x.z);
            df_add_prod(s, a.w, x.w);
        }
        for (int k = (n4 << 2) + lane; k < N; k += 32) df_add_prod(s, Ai[k], u[k]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            DF t;
            t.hi = __shfl_xor_sync(0xffffffffu, s.hi, o);
            t.lo = __shfl_xor_sync(0xffffffffu, s.lo, o);
            s = df_add(s, t);
        }
        if (lane == 0) {
            // r_i = b_i - (hi + lo), rounded once to single
            float ri;
            if (b) {
                float d, e;
                two_sum(b[i], -s.hi, d, e);
                ri = __fadd_rn(d, __fsub_rn(e, s.lo));
            } else {
                ri = __fadd_rn(s.hi, s.lo);
            }
            r[i] = ri;
            sq = (double)ri * (double)ri;
        }
    }
    return sq;
}

__global__ void __launch_bounds__(kGemvWarps * 32)
    k_gemv_residual(int N, const float* __restrict__ A, int64_t ld, const float* __restrict__ b,
                    const float* __restrict__ u, float* __restrict__ r, double* __restrict__ partial,
                    unsigned* __restrict__ counter, double* __restrict__ rnorm)
{
    __shared__ double red[kGemvWarps];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * kGemvWarps + warp;
    const double sq = (i < N) ? gemv_row(N, A, ld, b, u, r, i, lane) : 0.0;
    if (lane == 0) red[warp] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < kGemvWarps; ++q) t += red[q];
        partial[blockIdx.x] = t;
        __threadfence();
        unsigned done = atomicAdd(counter, 1u);
        last = (done == gridDim.x - 1);
    }
    __syncthreads();
    if (last && rnorm) {
        __shared__ double buf[kGemvWarps * 32];
        __threadfence();
        const double t = ordered_sum_staged(partial, (int)gridDim.x, buf);
        if (threadIdx.x == 0) *rnorm = sqrt(t);
    }
    if (last && threadIdx.x == 0) *counter = 0u;
}

int gemv_partials(int N) { return (int)cdiv(N, kGemvWarps); }

// Grouped residual r = b - J32 u: one block per task {instance, first row},
// instances with an IR step in progress only; per-instance block partials
// summed in block order by the instance's last block (into st.nr_new).
__global__ void __launch_bounds__(kGemvWarps * 32)
    k_gemv_residual_g(const BInst* __restrict__ inst, BState* __restrict__ st, const BTask* __restrict__ tasks)
{
    __shared__ double red[kGemvWarps];
    __shared__ bool last;
    const BTask tk = tasks[blockIdx.x];
    const BInst& I = inst[tk.inst];
    BState& S = st[tk.inst];
    if (S.status != BS_ACTIVE || !S.lin_active) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int N = I.N, i = tk.i0 + warp;
    const double sq = (i < N) ? gemv_row(N, I.J32, I.ld, I.b, I.u, I.r, i, lane) : 0.0;
    if (lane == 0) red[warp] = sq;
    __syncthreads();
    const int blk = tk.i0 / kGemvWarps, nblk = (N + kGemvWarps - 1) / kGemvWarps;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < kGemvWarps; ++q) t += red[q];
        I.part[blk] = t;
        __threadfence();
        last = (atomicAdd(&I.cnt[1], 1u) == (unsigned)(nblk - 1));
    }
    __syncthreads();
    if (last) {
        __shared__ double buf[kGemvWarps * 32];
        __threadfence();
        const double t = ordered_sum_staged(I.part, nblk, buf);
        if (threadIdx.x == 0) {
            S.nr_new = sqrt(t);
            I.cnt[1] = 0u;
        }
    }
}

int gemv_block_rows() { return kGemvWarps; }

nl_status launch_gemv_residual_g(const BInst* inst, BState* st, const BTask* tasks, int ntasks, cudaStream_t st_)
{
    if (ntasks <= 0) return NL_OK;
    prof_begin("k_gemv_residual", st_);
    k_gemv_residual_g<<<(unsigned)ntasks, kGemvWarps * 32, 0, st_>>>(inst, st, tasks);
    prof_end("k_gemv_residual", st_);
    NL_CUDA_OK(cudaGetLastError());
    return NL_OK;
}

nl_status launch_gemv_residual(int N, const float* A, int64_t ld, const float* b, const float* u, float* r,
                               double* partial, unsigned* counter, double* rnorm, cudaStream_t st)
{
    if ((ld & 3) || (((uintptr_t)A) & 15) || (((uintptr_t)u) & 15)) {
        set_error("gemv: A rows and u must be 16-byte aligned (ld multiple of 4)");
        return NL_EINVAL;
    }
    prof_begin("k_gemv_residual", st);
    k_gemv_residual<<<(unsigned)cdiv(N, kGemvWarps), kGemvWarps * 32, 0, st>>>(N, A, ld, b, u, r, partial, counter,
                                                                              rnorm);
    prof_end("k_gemv_residual", st);
    NL_CUDA_OK(cudaGetLastError());
    return NL_OK;
}

// ||v||_2 of a single vector (double accumulation of squares).
__global__ void __launch_bounds__(256) k_norm32(int N, const float* __restrict__ v, double* __restrict__ partial,
                                                unsigned* __restrict__ counter, double* __restrict__ out)
{
    __shared__ double red[8];
    __shared__ bool last;
    double s = 0.0;
    for (int i = blockIdx.x * 256 + threadIdx.x; i < N; i += gridDim.x * 256) s += (double)v[i] * (double)v[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = s;
        __threadfence();
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (last) {
        __shared__ double buf[256];
        __threadfence();
        const double t = ordered_sum_staged(partial, (int)gridDim.x, buf);
        if (threadIdx.x == 0) {
            *out = sqrt(t);
            *counter = 0u;
        }
    }
}

nl_status launch_norm32(int N, const float* v, double* partial, unsigned* counter, double* out, cudaStream_t st)
{
    int grid = (int)std::min<int64_t>(cdiv(N, 256), 64);
    k_norm32<<<grid, 256, 0, st>>>(N, v, partial, counter, out);
    NL_CUDA_OK(cudaGetLastError());
    return NL_OK;
}

// b = I_d^s(-F / ||F||), eq. (2.17), and the double variant.
__global__ void k_scale_rhs32(int N, const double* __restrict__ F, const double* __restrict__ fnorm,
                              float* __restrict__ b)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) b[i] = (float)(-F[i] / *fnorm);
}
__global__ void k_scale_rhs64(int N, const double* __restrict__ F, const double* __restrict__ fnorm,
                              double* __restrict__ b)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) b[i] = -F[i] / *fnorm;
}

nl_status launch_scale_rhs32(int N, const double* F, const double* fnorm, float* b, cudaStream_t st)
{
    k_scale_rhs32<<<(unsigned)cdiv(N, 256), 256, 0, st>>>(N, F, fnorm, b);
    NL_CUDA_OK(cudaGetLastError());
    return NL_OK;
}
nl_status launch_scale_rhs64(int N, const double* F, const double* fnorm, double* b, cudaStream_t st)
{
    k_scale_rhs64<<<(unsigned)cdiv(N, 256), 256, 0, st>>>(N, F, fnorm, b);
    NL_CUDA_OK(cudaGetLastError());
    return NL_OK;
}

__global__ void k_axpy32(int N, float a, const float* __restrict__ x, float* __restrict__ y)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) y[i] = fmaf(a, x[i], y[i]);
}

nl_status launch_axpy32(int N, float a, const float* x, float* y, cudaStream_t st)
{
    k_axpy32<<<(unsigned)cdiv(N, 256), 256, 0, st>>>(N, a, x, y);
    NL_CUDA_OK(cudaGetLastError());
    return NL_OK;
}

// ----------------------------------------------------------------- GMRES --
// ws layout (doubles): H[(m+1) x m] row-major | cs[m] | sn[m] | g[m+1] |
//                      scal[4] = {beta, residual estimate, breakdown, unused}
__host__ __device__ inline int ws_cs(int m) { return (m + 1) * m; }
__host__ __device__ inline int ws_sn(int m) { return ws_cs(m) + m; }
__host__ __device__ inline int ws_g(int m) { return ws_sn(m) + m; }
__host__ __device__ inline int ws_scal(int m) { return ws_g(m) + m + 1; }

int gmres_ws_doubles(int m) { return ws_scal(m) + 4; }
int gmres_scal_offset(int m) { return ws_scal(m); }

constexpr int kGmresThreads = 1024;

// V_0 = z / ||z||, g = ||z|| e_1.
__global__ void __launch_bounds__(kGmresThreads) k_gmres_start(int N, const float* __restrict__ z,
                                                               float* __restrict__ V, double* __restrict__ ws, int m)
{
    __shared__ float red[kGmresThreads / 32];
    float s = 0.0f;
    for (int i = threadIdx.x; i < N; i += kGmresThreads) s = fmaf(z[i], z[i], s);
    s = block_sum(s, red);
    const float beta = sqrtf(s);
    const float inv = (beta > 0.0f) ? 1.0f / beta : 0.0f;
    for (int i = threadIdx.x; i < N; i += kGmresThreads) V[i] = z[i] * inv;
    double* g = ws + ws_g(m);
    for (int k = threadIdx.x; k <= m; k += kGmresThreads) g[k] = (k == 0) ? (double)beta : 0.0;
    if (threadIdx.x == 0) {
        double* sc = ws + ws_scal(m);
        sc[0] = beta;
        sc[1] = beta;
        sc[2] = 0.0;
    }
}

nl_status launch_gmres_start(int N, const float* z, float* V, double* ws, int m, cudaStream_t st)
{
    k_gmres_start<<<1, kGmresThreads, 0, st>>>(N, z, V, ws, m);
    NL_CUDA_OK(cudaGetLastError());
    return NL_OK;
}

// Arnoldi step j (0-based): w = M^{-1} A v_j is given; modified Gram-Schmidt
// against v_0..v_j, h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j}; then the
// previous Givens rotations are applied to column j, a new one zeroes
// h_{j+1,j}, and g is updated; |g_{j+1}| is the residual estimate.
__global__ void __launch_bounds__(kGmresThreads) k_arnoldi(int N, int64_t ldv, float* __restrict__ w, float* __restrict__ V,
                                                           int j, double* __restrict__ ws, int m)
{
    __shared__ float red[kGmresThreads / 32];
    __shared__ double hcol[64];
    for (int i = 0; i <= j; ++i) {
        const float* vi = V + (int64_t)i * ldv;
        float s = 0.0f;
        for (int k = threadIdx.x; k < N; k += kGmresThreads) s = fmaf(w[k], vi[k], s);
        s = block_sum(s, red);
        for (int k = threadIdx.x; k < N; k += kGmresThreads) w[k] = fmaf(-s, vi[k], w[k]);
        if (threadIdx.x == 0) hcol[i] = s;
    }
    float s = 0.0f;
    for (int k = threadIdx.x; k < N; k += kGmresThreads) s = fmaf(w[k], w[k], s);
    s = block_sum(s, red);
    const float hn = sqrtf(s);
    const float inv = (hn > 0.0f) ? 1.0f / hn : 0.0f;
    float* vn = V + (int64_t)(j + 1) * ldv;
    for (int k = threadIdx.x; k < N; k += kGmresThreads) vn[k] = w[k] * inv;
    if (threadIdx.x == 0) {
        double* H = ws;
        double* cs = ws + ws_cs(m);
        double* sn = ws + ws_sn(m);
        double* g = ws + ws_g(m);
        double* sc = ws + ws_scal(m);
        hcol[j + 1] = hn;
        for (int i = 0; i < j; ++i) {
            double a = hcol[i], b = hcol[i + 1];
            hcol[i] = cs[i] * a + sn[i] * b;
            hcol[i + 1] = -sn[i] * a + cs[i] * b;
        }
        double a = hcol[j], b = hcol[j + 1];
        double rho = hypot(a, b);
        cs[j] = (rho == 0.0) ? 1.0 : a / rho;
        sn[j] = (rho == 0.0) ? 0.0 : b / rho;
        hcol[j] = rho;
        hcol[j + 1] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        for (int i = 0; i <= j + 1; ++i) H[i * m + j] = hcol[i];
        sc[1] = fabs(g[j + 1]);
        sc[2] = (hn == 0.0f) ? 1.0 : 0.0;
    }
}

nl_status launch_arnoldi(int N, int64_t ldv, float* w, float* V, int j, double* ws, int m, cudaStream_t st)
{
    if (m > 62) {
        set_error("GMRES restart length %d exceeds 62", m);
        return NL_EINVAL;
    }
    k_arnoldi<<<1, kGmresThreads, 0, st>>>(N, ldv, w, V, j, ws, m);
    NL_CUDA_OK(cudaGetLastError());
    return NL_OK;
}

// d += V y with y = R^{-1} g over the first jcols columns (R upper triangle of H).
__global__ void __launch_bounds__(256) k_gmres_update(int N, int64_t ldv, const float* __restrict__ V,
                                                      const double* __restrict__ ws, int m, int jcols,
                                                      float* __restrict__ d)
{
    __shared__ float ys[64];
    if (threadIdx.x == 0) {
        const double* H = ws;
        const double* g = ws + ws_g(m);
        double y[64];
        for (int i = jcols - 1; i >= 0; --i) {
            double s = g[i];
            for (int k = i + 1; k < jcols; ++k) s -= H[i * m + k] * y[k];
            y[i] = s / H[i * m + i];
        }
        for (int i = 0; i < jcols; ++i) ys[i] = (float)y[i];
    }
    __syncthreads();
    int q = blockIdx.x * 256 + threadIdx.x;
    if (q < N) {
        float acc = d[q];
        for (int k = 0; k < jcols; ++k) acc = fmaf(ys[k], V[(int64_t)k * ldv + q], acc);
        d[q] = acc;
    }
}

nl_status launch_gmres_update(int N, int64_t ldv, const float* V, double* ws, int m, int jcols, float* d,
                              cudaStream_t st)
{
    if (jcols <= 0) return NL_OK;
    k_gmres_update<<<(unsigned)cdiv(N, 256), 256, 0, st>>>(N, ldv, V, ws, m, jcols, d);
    NL_CUDA_OK(cudaGetLastError());
    return NL_OK;
}

}  // namespace nl
