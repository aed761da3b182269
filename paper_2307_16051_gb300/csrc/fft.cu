// fft.cu — the residual of eq. (3.2) in O(N log N) with a fast Fourier
// transform (Section 3: F can be evaluated with an FFT; the Jacobian stays
// analytic).
//
// With 0-based indices the sum of eq. (3.2) is a Hankel product,
//   y_i = sum_j x_j h[i+j],  h[k] = 1/(k+1),  t_i = c/(2N) (i + 1/2) y_i.
// Reversing x (z_m = x_{N-1-m}) turns it into the convolution
//   y_i = (h * z)[i + N - 1],
// and a circular convolution of length L >= 2N gives the same values at the
// indices N-1 .. 2N-2 (a wrapped term would need an index sum of at least
// L + N - 1 > 3N - 3, the largest that occurs).  So one forward transform of z,
// a product with the transform of h (computed once per N), and one inverse
// transform give every y_i, in double precision.
//
// The transforms are hand-written: a four-step split L = L1 L2 (L a power of
// two, L1 <= L2 <= 256) into two launches, each CTA doing one radix-2
// Stockham transform of length L1 or L2 in shared memory,
//   pass A: for each n2, Y[n2][k1] = w_L^(n2 k1) sum_n1 x[L2 n1 + n2] w_L1^(n1 k1),
//   pass B: for each k1, X[k1 + L1 k2] = sum_n2 Y[n2][k1] w_L2^(n2 k2),
// with twiddles w_L^k = exp(-2 pi i k / L) from a table made once with
// sincospi.  The inverse transform is the forward one applied to the
// conjugate (only its real part is needed).  The Newton update x + ||F|| u
// is fused into the first pass, the residual, r and the deterministic norm
// into the last, so one evaluation is four launches.
#include "common.cuh"
#include "internal.h"

namespace nl {

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__global__ void k_fft_twiddles(int L, double2* __restrict__ tw)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < L) {
        double s, c;
        sincospi(2.0 * (double)k / (double)L, &s, &c);
        tw[k] = make_double2(c, -s);
    }
}

// Radix-2 Stockham transform of length n (a power of two) held in A, with B
// as the ping-pong buffer; returns the buffer that holds the result.  Stage
// with half-size Ls: thread j combines entries j and j + n/2 into positions
// 2 Ls (j / Ls) + j % Ls and that + Ls, with the twiddle w_(2 Ls)^(j % Ls).
__device__ __forceinline__ double2* dft_smem(double2* A, double2* B, int n, int L, const double2* __restrict__ tw)
{
    const int half = n >> 1;
    for (int Ls = 1; Ls < n; Ls <<= 1) {
        const int stride = L / (2 * Ls);
        for (int j = threadIdx.x; j < half; j += blockDim.x) {
            const int k = j & (Ls - 1), p = j / Ls;
            const double2 w = tw[k * stride];
            const double2 a = A[j];
            const double2 b = cmul(A[j + half], w);
            B[p * 2 * Ls + k] = make_double2(a.x + b.x, a.y + b.y);
            B[p * 2 * Ls + k + Ls] = make_double2(a.x - b.x, a.y - b.y);
        }
        __syncthreads();
        double2* t = A;
        A = B;
        B = t;
    }
    return A;
}

// Pass A.  MODE 0: the input is `in` (length L, natural order).  MODE 1: the
// input is z_m = v_(N-1-m) for m < N (0 beyond), v = x + scale u (the Newton
// update, rounded as in the direct residual), u may be NULL.
template <int MODE, typename TU>
__global__ void __launch_bounds__(128) k_fft_pass_a(int N, int L, int L1, int L2, const double2* __restrict__ tw,
                                                    const double2* __restrict__ in, const double* __restrict__ x,
                                                    const TU* __restrict__ u, double scale, double2* __restrict__ Y)
{
    extern __shared__ double2 fsm[];
    const int n2 = blockIdx.x;
    for (int n1 = threadIdx.x; n1 < L1; n1 += blockDim.x) {
        const int m = L2 * n1 + n2;
        double2 v;
        if constexpr (MODE == 0) {
            v = in[m];
        } else {
            double val = 0.0;
            if (m < N) {
                const int j = N - 1 - m;
                val = x[j];
                if (u) val = __dadd_rn(val, __dmul_rn(scale, (double)u[j]));
            }
            v = make_double2(val, 0.0);
        }
        fsm[n1] = v;
    }
    __syncthreads();
    const double2* R = dft_smem(fsm, fsm + L1, L1, L, tw);
    for (int k1 = threadIdx.x; k1 < L1; k1 += blockDim.x) Y[n2 * L1 + k1] = cmul(R[k1], tw[n2 * k1]);
}

// Pass B.  MODE 0: out = X.  MODE 1: out = conj(X * Hh) (the input of the
// inverse transform).  MODE 2: the inverse transform's real part / L at the
// indices N-1 .. 2N-2 gives y_i; then t_i, r_i = 1/(1 - t_i), F_i = v_i - r_i
// (v = x + scale u, also written to xout when given), and ||F||_2 with a
// deterministic reduction (per-block partials, the last block sums them in
// block order).
template <int MODE, typename TU>
__global__ void __launch_bounds__(128) k_fft_pass_b(int N, int L, int L1, int L2, const double2* __restrict__ tw,
                                                    const double2* __restrict__ Y, const double2* __restrict__ Hh,
                                                    double2* __restrict__ out, double c, const double* __restrict__ x,
                                                    const TU* __restrict__ u, double scale, double* __restrict__ xout,
                                                    double* __restrict__ F, double* __restrict__ rr,
                                                    double* __restrict__ part, unsigned* __restrict__ cnt,
                                                    double* __restrict__ fnorm)
{
    extern __shared__ double2 fsm[];
    __shared__ double red[4];
    __shared__ bool last;
    const int k1 = blockIdx.x;
    for (int n2 = threadIdx.x; n2 < L2; n2 += blockDim.x) fsm[n2] = Y[n2 * L1 + k1];
    __syncthreads();
    const double2* R = dft_smem(fsm, fsm + L2, L2, L, tw);
    if constexpr (MODE == 0) {
        for (int k2 = threadIdx.x; k2 < L2; k2 += blockDim.x) out[k1 + L1 * k2] = R[k2];
    } else if constexpr (MODE == 1) {
        for (int k2 = threadIdx.x; k2 < L2; k2 += blockDim.x) {
            const int m = k1 + L1 * k2;
            const double2 p = cmul(R[k2], Hh[m]);
            out[m] = make_double2(p.x, -p.y);
        }
    } else {
        double acc = 0.0;
        const double invL = 1.0 / (double)L;
        for (int k2 = threadIdx.x; k2 < L2; k2 += blockDim.x) {
            const int m = k1 + L1 * k2;
            if (m >= N - 1 && m <= 2 * N - 2) {
                const int i = m - (N - 1);
                const double s = R[k2].x * invL;
                const double t = c / (2.0 * (double)N) * ((double)i + 0.5) * s;
                const double ri = 1.0 / (1.0 - t);
                double xi = x[i];
                if (u) xi = __dadd_rn(xi, __dmul_rn(scale, (double)u[i]));
                const double fi = xi - ri;
                if (xout) xout[i] = xi;
                F[i] = fi;
                rr[i] = ri;
                acc += fi * fi;
            }
        }
        // deterministic block sum (blockDim.x <= 128: four warps)
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = 0.0;
            for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) b += red[w];
            part[k1] = b;
            __threadfence();
            last = (atomicAdd(cnt, 1u) == (unsigned)(L1 - 1));
        }
        __syncthreads();
        if (last) {
            __shared__ double buf[128];
            __threadfence();
            const double sum = ordered_sum_staged(part, L1, buf);
            if (threadIdx.x == 0) {
                *fnorm = sqrt(sum);
                *cnt = 0u;
            }
        }
    }
}

__global__ void k_fft_hpad(int N, int L, double2* __restrict__ out)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < L) out[m] = make_double2(m < 2 * N - 1 ? 1.0 / (double)(m + 1) : 0.0, 0.0);
}

static void fft_sizes(int N, int* L, int* L1, int* L2)
{
    int l = 4;
    while (l < 2 * N) l <<= 1;
    int lg = 0;
    while ((1 << lg) < l) ++lg;
    *L = l;
    *L1 = 1 << (lg / 2);
    *L2 = l / *L1;
}

size_t fft_work_bytes(int N)
{
    int L, L1, L2;
    fft_sizes(N, &L, &L1, &L2);
    return 4 * round_up((size_t)L * sizeof(double2), 256) + round_up((size_t)L1 * sizeof(double), 256) + 256;
}

void fft_work_carve(void* base, int N, FftPlan* p)
{
    fft_sizes(N, &p->L, &p->L1, &p->L2);
    p->N = N;
    char* q = (char*)base;
    const size_t cb = round_up((size_t)p->L * sizeof(double2), 256);
    p->tw = (double2*)q;
    q += cb;
    p->Hh = (double2*)q;
    q += cb;
    p->Y = (double2*)q;
    q += cb;
    p->V = (double2*)q;
    q += cb;
    p->part = (double*)q;
    q += round_up((size_t)p->L1 * sizeof(double), 256);
    p->cnt = (unsigned*)q;
}

static unsigned fft_threads(int n) { return (unsigned)std::max(32, std::min(128, n / 2)); }

nl_status fft_prepare(const FftPlan& p, cudaStream_t st)
{
    const int L = p.L, L1 = p.L1, L2 = p.L2;
    NL_CUDA_OK(cudaMemsetAsync(p.cnt, 0, sizeof(unsigned), st));
    k_fft_twiddles<<<(unsigned)cdiv(L, 256), 256, 0, st>>>(L, p.tw);
    k_fft_hpad<<<(unsigned)cdiv(L, 256), 256, 0, st>>>(p.N, L, p.V);
    k_fft_pass_a<0, double><<<L2, fft_threads(L1), 2 * L1 * sizeof(double2), st>>>(p.N, L, L1, L2, p.tw, p.V, nullptr,
                                                                                   nullptr, 0.0, p.Y);
    k_fft_pass_b<0, double><<<L1, fft_threads(L2), 2 * L2 * sizeof(double2), st>>>(
        p.N, L, L1, L2, p.tw, p.Y, nullptr, p.Hh, 0.0, nullptr, nullptr, 0.0, nullptr, nullptr, nullptr, nullptr,
        nullptr, nullptr);
    NL_CUDA_OK(cudaGetLastError());
    return NL_OK;
}

template <typename TU>
static nl_status residual_fft_t(const FftPlan& p, double c, const double* x, const TU* u, double scale, double* xout,
                                double* F, double* rr, double* fnorm, cudaStream_t st)
{
    const int N = p.N, L = p.L, L1 = p.L1, L2 = p.L2;
    const size_t s1 = 2 * L1 * sizeof(double2), s2 = 2 * L2 * sizeof(double2);
    prof_begin("k_fft", st);
    k_fft_pass_a<1, TU><<<L2, fft_threads(L1), s1, st>>>(N, L, L1, L2, p.tw, nullptr, x, u, scale, p.Y);
    k_fft_pass_b<1, TU><<<L1, fft_threads(L2), s2, st>>>(N, L, L1, L2, p.tw, p.Y, p.Hh, p.V, 0.0, nullptr, nullptr,
                                                          0.0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    k_fft_pass_a<0, TU><<<L2, fft_threads(L1), s1, st>>>(N, L, L1, L2, p.tw, p.V, nullptr, nullptr, 0.0, p.Y);
    k_fft_pass_b<2, TU><<<L1, fft_threads(L2), s2, st>>>(N, L, L1, L2, p.tw, p.Y, nullptr, nullptr, c, x, u, scale,
                                                          xout, F, rr, p.part, p.cnt, fnorm);
    prof_end("k_fft", st);
    NL_CUDA_OK(cudaGetLastError());
    return NL_OK;
}

nl_status launch_residual_fft(const FftPlan& p, double c, const double* x, const void* u, int u_is_double,
                              double scale, double* xout, double* F, double* rr, double* fnorm, cudaStream_t st)
{
    if (u_is_double) return residual_fft_t<double>(p, c, x, (const double*)u, scale, xout, F, rr, fnorm, st);
    return residual_fft_t<float>(p, c, x, (const float*)u, scale, xout, F, rr, fnorm, st);
}

}  // namespace nl
