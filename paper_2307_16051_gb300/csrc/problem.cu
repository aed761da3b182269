// problem.cu — the H-equation residual (fused with the Newton update) and
// the analytic Jacobian, Section 3 eq. (3.2).
//
// With 0-based i, j the kernel entry is mu_i/(mu_j+mu_i) = (i+1/2)/(i+j+1),
// so the sum of eq. (3.2) is a Hankel matrix-vector product
//   t_i = c/(2N) (i + 1/2) sum_j x_j h[i+j],   h[k] = 1/(k+1),
// evaluated from a 2N-1 entry table of reciprocals: no N x N matrix is read.
#include "common.cuh"
#include "internal.h"

namespace nl {

// ---------------------------------------------------------------- K1: F(x) --
// Block = kFRows rows x kFSlices j-slices; rows and j-chunks are staged in
// shared memory (x + scale*u for the chunk, and the h window it needs).
constexpr int kFRows = 32, kFSlices = 8, kFChunk = 256;

// Rows [i0, i0 + kFRows) of F at x + scale u (u may be NULL); returns the
// block's sum of F_i^2 (valid in every thread).
template <typename TU>
__device__ __forceinline__ double residual_rows(int N, double c, const double* __restrict__ x,
                                                const TU* __restrict__ u, double scale,
                                                const double* __restrict__ htab, double* __restrict__ xout,
                                                double* __restrict__ F, double* __restrict__ rr, int i0)
{
    __shared__ double xs[kFChunk];
    __shared__ double hw[kFChunk + kFRows];
    __shared__ double red[kFSlices][kFRows + 1];
    __shared__ double bsum;
    const int r = threadIdx.x % kFRows, q = threadIdx.x / kFRows;
    const int i = i0 + r;
    double acc = 0.0;
    for (int j0 = 0; j0 < N; j0 += kFChunk) {
        __syncthreads();
        for (int t = threadIdx.x; t < kFChunk; t += blockDim.x) {
            int j = j0 + t;
            double v = 0.0;
            if (j < N) {
                v = x[j];
                // x + ||F|| u: a product and a sum, each rounded (eq. (2.18))
                if (u) v = __dadd_rn(v, __dmul_rn(scale, (double)u[j]));
            }
            xs[t] = v;
        }
        for (int t = threadIdx.x; t < kFChunk + kFRows; t += blockDim.x) {
            int k = i0 + j0 + t;
            hw[t] = (k < 2 * N - 1) ? htab[k] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int jj = q; jj < kFChunk; jj += kFSlices) acc = fma(xs[jj], hw[r + jj], acc);
    }
    red[q][r] = acc;
    __syncthreads();
    double f2 = 0.0;
    if (q == 0 && i < N) {
        double s = 0.0;
        for (int k = 0; k < kFSlices; ++k) s += red[k][r];
        double t = c / (2.0 * (double)N) * ((double)i + 0.5) * s;
        double ri = 1.0 / (1.0 - t);
        double xi = x[i];
        if (u) xi = __dadd_rn(xi, __dmul_rn(scale, (double)u[i]));
        double fi = xi - ri;
        if (xout) xout[i] = xi;
        F[i] = fi;
        rr[i] = ri;
        f2 = fi * fi;
    }
    // deterministic norm: per-block partial, the last block sums them in order
    __syncthreads();
    if (q == 0) {
        double v = f2;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (r == 0) bsum = v;
    }
    __syncthreads();
    return bsum;
}

template <typename TU>
__global__ void __launch_bounds__(kFRows* kFSlices)
    k_residual(int N, double c, const double* __restrict__ x, const TU* __restrict__ u, double scale,
               const double* __restrict__ htab, double* __restrict__ xout, double* __restrict__ F,
               double* __restrict__ rr, double* __restrict__ partial, unsigned* __restrict__ counter,
               double* __restrict__ fnorm)
{
    __shared__ bool last;
    const double v = residual_rows<TU>(N, c, x, u, scale, htab, xout, F, rr, blockIdx.x * kFRows);
    if (threadIdx.x == 0) partial[blockIdx.x] = v;
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned done = atomicAdd(counter, 1u);
        last = (done == gridDim.x - 1);
    }
    __syncthreads();
    if (last) {
        __shared__ double buf[kFRows * kFSlices];
        __threadfence();
        const double s = ordered_sum_staged(partial, (int)gridDim.x, buf);
        if (threadIdx.x == 0) {
            *fnorm = sqrt(s);
            *counter = 0u;
        }
    }
}

__global__ void k_htab(int N, double* htab)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < 2 * N - 1) htab[k] = 1.0 / (double)(k + 1);
}

nl_status launch_htab(int N, double* htab, cudaStream_t st)
{
    k_htab<<<(unsigned)cdiv(2 * (int64_t)N, 256), 256, 0, st>>>(N, htab);
    NL_CUDA_OK(cudaGetLastError());
    return NL_OK;
}

nl_status launch_residual(int N, double c, const double* x, const void* u, int u_is_double, double scale,
                          const double* htab, double* xout, double* F, double* rr, double* partial,
                          unsigned* counter, double* fnorm, cudaStream_t st)
{
    unsigned grid = (unsigned)cdiv(N, kFRows);
    prof_begin("k_residual", st);
    if (u_is_double)
        k_residual<double><<<grid, kFRows * kFSlices, 0, st>>>(N, c, x, (const double*)u, scale, htab, xout, F,
                                                               rr, partial, counter, fnorm);
    else
        k_residual<float><<<grid, kFRows * kFSlices, 0, st>>>(N, c, x, (const float*)u, scale, htab, xout, F,
                                                              rr, partial, counter, fnorm);
    prof_end("k_residual", st);
    NL_CUDA_OK(cudaGetLastError());
    return NL_OK;
}

int residual_partials(int N) { return (int)cdiv(N, kFRows); }

// Grouped residual: one block per task {instance, first row}.  Per-instance
// block partials are summed in block order by the instance's last block.
__global__ void __launch_bounds__(kFRows* kFSlices)
    k_residual_g(const BInst* __restrict__ inst, BState* __restrict__ st, const BTask* __restrict__ tasks, int mode,
                 const double* __restrict__ htab)
{
    __shared__ bool last;
    const BTask tk = tasks[blockIdx.x];
    const BInst& I = inst[tk.inst];
    BState& S = st[tk.inst];
    if (mode != 0 && S.status != BS_ACTIVE) return;
    const int N = I.N;
    const int par = (mode == 0) ? 0 : S.par;
    const double* x = I.x[par];
    double v;
    if (mode == 0)
        v = residual_rows<float>(N, I.c, x, nullptr, 0.0, htab, nullptr, I.F, I.rr, tk.i0);
    else if (mode == 1)
        v = residual_rows<float>(N, I.c, x, I.u, S.fn, htab, I.x[par ^ 1], I.F, I.rr, tk.i0);
    else
        v = residual_rows<double>(N, I.c, x, I.u64, S.fn, htab, I.x[par ^ 1], I.F, I.rr, tk.i0);
    const int blk = tk.i0 / kFRows, nblk = (N + kFRows - 1) / kFRows;
    if (threadIdx.x == 0) {
        I.part[blk] = v;
        __threadfence();
        last = (atomicAdd(&I.cnt[0], 1u) == (unsigned)(nblk - 1));
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += __ldcg(&I.part[b]);
        S.fn = sqrt(s);
        I.cnt[0] = 0u;
    }
}

int residual_block_rows() { return kFRows; }

nl_status launch_residual_g(const BInst* inst, BState* st, const BTask* tasks, int ntasks, int mode,
                            const double* htab, cudaStream_t st_)
{
    if (ntasks <= 0) return NL_OK;
    k_residual_g<<<(unsigned)ntasks, kFRows * kFSlices, 0, st_>>>(inst, st, tasks, mode, htab);
    NL_CUDA_OK(cudaGetLastError());
    return NL_OK;
}

// ------------------------------------------------------- K2: the Jacobian --
// J_ij = delta_ij - w_i h[i+j],  w_i = c/(2N) r_i^2 (i + 1/2).  Each thread
// writes 8 consecutive columns of one row: two 16-byte stores of J32 and one
// of J16.  w_i is formed in double and rounded to single; the product with
// the single-rounded h[i+j] and the subtraction are one single-precision FMA.
constexpr int kJCols = 8;

// One CTA per 256 columns x 32 rows: the 287 Hankel entries the tile needs are
// converted to single once into shared memory, and each row's factor
// w_i = c/(2N) r_i^2 (i + 1/2) once per row; every thread then writes its
// column of the 32 rows (coalesced rows of J32 and J16).  Per entry the value
// is fma(-w_i, fl32(h_{i+j}), [i == j]), rounded once more for J16.
//
// Optional scaling into the binary16 range (rs != NULL): J16 row i is
// fl16(2^k_i J32_ij), where 2^k_i is the largest power of two with
// 2^k_i B_i <= 2^13 for the row bound B_i = 1 + c/(2N) r_i^2 >= max_j |J_ij|
// (|J_ij| <= delta_ij + c/(2N) r_i^2 mu_i/(mu_i+mu_j), mu_i/(mu_i+mu_j) < 1);
// k_i = 13 - ceil(log2 B_i) exactly, from frexp.  The product with 2^k_i is
// exact in single precision; the factor goes to rs[i] for the solves.
constexpr int kJRows = 32;

__device__ __forceinline__ float row_scale16(int N, double c, double ri)
{
    const double B = 1.0 + (c / (2.0 * (double)N)) * ri * ri;
    int e;
    const double m = frexp(B, &e);
    return ldexpf(1.0f, 13 - ((m == 0.5) ? e - 1 : e));
}

__global__ void __launch_bounds__(256) k_jacobian(int N, double c, const double* __restrict__ rr,
                                                  const double* __restrict__ htab, float* __restrict__ J32,
                                                  int64_t ld32, __half* __restrict__ J16, int64_t ld16,
                                                  int ldmax, float* __restrict__ rs)
{
    __shared__ float hw[256 + kJRows];
    __shared__ float wr[kJRows];
    __shared__ float sr[kJRows];
    const int i0 = blockIdx.y * kJRows, j0 = blockIdx.x * 256;
    for (int q = threadIdx.x; q < 256 + kJRows; q += 256) {
        const int k = i0 + j0 + q;
        hw[q] = (k < 2 * N - 1) ? (float)htab[k] : 0.0f;
    }
    if (threadIdx.x < kJRows) {
        const int i = i0 + threadIdx.x;
        float w = 0.0f, sc = 1.0f;
        if (i < N) {
            const double ri = rr[i];
            w = (float)(c / (2.0 * (double)N) * ri * ri * ((double)i + 0.5));
            if (rs) {
                sc = row_scale16(N, c, ri);
                if (blockIdx.x == 0) rs[i] = sc;
            }
        }
        wr[threadIdx.x] = w;
        sr[threadIdx.x] = sc;
    }
    __syncthreads();
    const int j = j0 + threadIdx.x;
    if (j >= ldmax) return;
    const int rows = min(kJRows, N - i0);
    for (int r = 0; r < rows; ++r) {
        const int i = i0 + r;
        const float e = (j < N) ? fmaf(-wr[r], hw[r + threadIdx.x], (i == j) ? 1.0f : 0.0f) : 0.0f;
        if (J32 && j < ld32) J32[(int64_t)i * ld32 + j] = e;
        if (J16 && j < ld16) J16[(int64_t)i * ld16 + j] = __float2half_rn(rs ? e * sr[r] : e);
    }
}

nl_status launch_jacobian(int N, double c, const double* rr, const double* htab, float* J32, int64_t ld32,
                          __half* J16, int64_t ld16, cudaStream_t st, float* rs)
{
    if ((J32 && (ld32 % kJCols)) || (J16 && (ld16 % kJCols))) {
        set_error("jacobian: leading dimensions must be multiples of %d", kJCols);
        return NL_EINVAL;
    }
    int ldmax = (int)std::max(J32 ? ld32 : 0, J16 ? ld16 : 0);
    dim3 grid((unsigned)cdiv(ldmax, 256), (unsigned)cdiv(N, kJRows));
    k_jacobian<<<grid, 256, 0, st>>>(N, c, rr, htab, J32, ld32, J16, ld16, ldmax, rs);
    NL_CUDA_OK(cudaGetLastError());
    return NL_OK;
}

__global__ void __launch_bounds__(256) k_jacobian64(int N, double c, const double* __restrict__ rr,
                                                    const double* __restrict__ htab, double* __restrict__ J,
                                                    int64_t ld)
{
    const int i = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ld) return;
    const double ri = rr[i];
    const double w = c / (2.0 * (double)N) * ri * ri * ((double)i + 0.5);
    J[(int64_t)i * ld + j] = (j < N) ? fma(-w, htab[i + j], (i == j) ? 1.0 : 0.0) : 0.0;
}

nl_status launch_jacobian64(int N, double c, const double* rr, const double* htab, double* J, int64_t ld,
                            cudaStream_t st)
{
    dim3 grid((unsigned)cdiv(ld, 256), (unsigned)N);
    k_jacobian64<<<grid, 256, 0, st>>>(N, c, rr, htab, J, ld);
    NL_CUDA_OK(cudaGetLastError());
    return NL_OK;
}

// Grouped Jacobian: one block per row of one instance (row_off gives the
// instance's first global row), the same arithmetic as k_jacobian /
// k_jacobian64.  Instances that are not BS_ACTIVE are skipped.
__global__ void __launch_bounds__(256) k_jacobian_g(const BInst* __restrict__ inst, const BState* __restrict__ st,
                                                    const int* __restrict__ row_off, int count,
                                                    const double* __restrict__ htab,
                                                    const float* __restrict__ htab32, int fp64)
{
    const int g = blockIdx.x;
    int lo = 0, hi = count - 1;  // last instance with row_off[k] <= g
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (row_off[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    const BInst& I = inst[lo];
    if (st[lo].status != BS_ACTIVE) return;
    const int i = g - row_off[lo], N = I.N;
    const double ri = I.rr[i];
    if (fp64) {
        const double w = I.c / (2.0 * (double)N) * ri * ri * ((double)i + 0.5);
        double* Ji = reinterpret_cast<double*>(I.J) + (int64_t)i * I.ld;
        for (int j = threadIdx.x; j < I.ld; j += blockDim.x)
            Ji[j] = (j < N) ? fma(-w, htab[i + j], (i == j) ? 1.0 : 0.0) : 0.0;
        return;
    }
    // the row factor once per row (double arithmetic), the Hankel entries from the single table
    __shared__ float wsh;
    if (threadIdx.x == 0) wsh = (float)(I.c / (2.0 * (double)N) * ri * ri * ((double)i + 0.5));
    __syncthreads();
    const float w = wsh;
    for (int j0 = threadIdx.x * kJCols; j0 < I.ld; j0 += blockDim.x * kJCols) {
        float v[kJCols];
#pragma unroll
        for (int t = 0; t < kJCols; ++t) {
            const int j = j0 + t;
            float e = 0.0f;
            if (j < N) e = fmaf(-w, htab32[i + j], (i == j) ? 1.0f : 0.0f);
            v[t] = e;
        }
        float4* p = reinterpret_cast<float4*>(I.J32 + (int64_t)i * I.ld + j0);
        p[0] = make_float4(v[0], v[1], v[2], v[3]);
        p[1] = make_float4(v[4], v[5], v[6], v[7]);
        __align__(16) __half h[kJCols];
#pragma unroll
        for (int t = 0; t < kJCols; ++t) h[t] = __float2half_rn(v[t]);
        *reinterpret_cast<uint4*>(reinterpret_cast<__half*>(I.J) + (int64_t)i * I.ld + j0) =
            *reinterpret_cast<uint4*>(h);
    }
}

nl_status launch_jacobian_g(const BInst* inst, const BState* st, const int* row_off, int count, int rows,
                            const double* htab, const float* htab32, int fp64, cudaStream_t st_)
{
    if (rows <= 0) return NL_OK;
    k_jacobian_g<<<(unsigned)rows, 256, 0, st_>>>(inst, st, row_off, count, htab, htab32, fp64);
    NL_CUDA_OK(cudaGetLastError());
    return NL_OK;
}

}  // namespace nl
