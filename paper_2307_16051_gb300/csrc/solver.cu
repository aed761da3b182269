// solver.cu — the Newton drivers and the C ABI (include/newton3p.h).
//
// Algorithm 1.1 [newton] / Algorithm 2.1 [newton3p]: evaluate F in double,
// tau = tau_r ||F(x0)|| + tau_a, and while ||F|| > tau: form the Jacobian,
// factor it, solve J s = -F with the scaled right-hand side of
// eqs. (2.17)-(2.18) (b = -F/||F||, s = ||F|| u), update x and re-evaluate F.
// The update x += s is fused into the next residual evaluation.
//
// Linear solvers (Section 2.2): IR (Algorithm IR) and GMRES-IR with the
// half-precision factors; success at ||b - J32 u|| <= eta ||b||, failure
// when the residual norm increases (the best iterate is kept), Section 3.1.
// Control runs on the host; each decision reads one device scalar back.
#include <atomic>
#include <chrono>
#include <type_traits>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace nl {

static thread_local char g_err[512] = "";

// Test hook (nl_debug_fail_allocs): the next g_fail_allocs device allocations
// of the library's handles fail as if the device were out of memory.
static std::atomic<int> g_fail_allocs{0};

cudaError_t dev_malloc(void** p, size_t bytes)
{
    int n = g_fail_allocs.load();
    while (n > 0) {
        if (g_fail_allocs.compare_exchange_weak(n, n - 1)) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
    }
    return cudaMalloc(p, bytes);
}

void set_error(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
const char* get_error() { return g_err; }

int num_sms()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// ---------------------------------------------------- per-kernel timing --
struct KernelTiming {
    std::mutex mu;
    std::string cls;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    int open = -1;
};
static KernelTiming g_kt;

void prof_begin(const char* kernel_class, cudaStream_t st)
{
    if (g_kt.cls.empty() || g_kt.cls != kernel_class) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    std::lock_guard<std::mutex> lock(g_kt.mu);
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return;
    cudaEventRecord(a, st);
    g_kt.ev.push_back({a, b});
    g_kt.open = (int)g_kt.ev.size() - 1;
}

void prof_end(const char* kernel_class, cudaStream_t st)
{
    if (g_kt.cls.empty() || g_kt.cls != kernel_class) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    std::lock_guard<std::mutex> lock(g_kt.mu);
    if (g_kt.open >= 0) cudaEventRecord(g_kt.ev[g_kt.open].second, st);
    g_kt.open = -1;
}

int set_max_dynamic_smem(const void* func)
{
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, func) != cudaSuccess ||
        cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes) !=
            cudaSuccess) {
        cudaError_t e = cudaGetLastError();
        set_error("cannot raise the dynamic shared-memory limit: %s", cudaGetErrorString(e));
        return NL_ECUDA;
    }
    return NL_OK;
}

__global__ void k_fill64(int N, double v, double* x)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) x[i] = v;
}


struct LinBufs {
    float *r, *d, *t, *w, *ubest, *V;
    int64_t ldv;
    double* gws;
    double* partial;
    unsigned* counter;
    double* dscal;  // device scalars: [0] norm(b), [1] residual norm
    // GMRES-IR preconditioner with a single-precision copy of the factors (null: on the fly)
    const float* LU32 = nullptr;
    const TrsvWork* tw32 = nullptr;
};

// M^{-1} v for GMRES-IR: the binary16 factors promoted on the fly, or their
// single-precision copy.
static nl_status precond_apply(int N, const __half* LU, int64_t ld16, const TrsvWork& tw, int& epoch, const float* v,
                               float* z, const LinBufs& B, cudaStream_t st, int* launches)
{
    if (B.LU32) return trsv_solve32(N, B.LU32, ld16, v, z, *B.tw32, ++epoch, st, launches);
    return trsv_solve16(N, LU, ld16, v, z, tw, ++epoch, st, launches);
}

struct LinResult {
    int iters = 0, outer = 0, failed = 0, converged = 0;
    double relres = 0.0;
};

struct Host {
    double* pin;  // pinned host scalars
    cudaStream_t st;
    int* launches;
    double read(const double* dev)
    {
        cudaMemcpyAsync(pin, dev, sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        return pin[0];
    }
    // *dev and a device error word in one synchronisation
    double read_err(const double* dev, const unsigned* err, unsigned* errv)
    {
        cudaMemcpyAsync(pin, dev, sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(pin + 4, err, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        memcpy(errv, pin + 4, sizeof(unsigned));
        return pin[0];
    }
    void read2(const double* dev, double* out)
    {
        cudaMemcpyAsync(pin, dev, 3 * sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        out[0] = pin[0];
        out[1] = pin[1];
        out[2] = pin[2];
    }
};

// Left-preconditioned restarted GMRES(m) from d0 = 0 for M^{-1} A d = M^{-1} r.
static nl_status gmres16(int N, const float* J32, int64_t ld32, const __half* LU, int64_t ld16, const TrsvWork& tw,
                         int& epoch, const float* r, float* d, int m, double gtol, int gcycles, LinBufs& B, Host& H,
                         int* steps_out)
{
    cudaStream_t st = H.st;
    const int so = gmres_scal_offset(m);
    int steps = 0;
    double beta0 = -1.0;
    NL_CUDA_OK(cudaMemsetAsync(d, 0, sizeof(float) * N, st));
    for (int cycle = 0; cycle < gcycles; ++cycle) {
        if (cycle == 0) {
            NL_CUDA_OK(cudaMemcpyAsync(B.t, r, sizeof(float) * N, cudaMemcpyDeviceToDevice, st));
        } else {
            NL_TRY(launch_gemv_residual(N, J32, ld32, r, d, B.t, B.partial, B.counter, nullptr, st));
            ++*H.launches;
        }
        NL_TRY(precond_apply(N, LU, ld16, tw, epoch, B.t, B.w, B, st, H.launches));
        NL_TRY(launch_gmres_start(N, B.w, B.V, B.gws, m, st));
        ++*H.launches;
        double sc[3];
        H.read2(B.gws + so, sc);
        const double beta = sc[0];
        if (beta0 < 0.0) beta0 = beta;
        if (beta == 0.0 || beta <= gtol * beta0) break;
        int jcols = 0;
        bool done = false;
        for (int j = 0; j < m; ++j) {
            NL_TRY(launch_gemv_residual(N, J32, ld32, nullptr, B.V + (int64_t)j * B.ldv, B.t, B.partial, B.counter,
                                        nullptr, st));
            NL_TRY(precond_apply(N, LU, ld16, tw, epoch, B.t, B.w, B, st, H.launches));
            NL_TRY(launch_arnoldi(N, B.ldv, B.w, B.V, j, B.gws, m, st));
            *H.launches += 2;
            H.read2(B.gws + so, sc);
            ++steps;
            jcols = j + 1;
            if (sc[1] <= gtol * beta0 || sc[2] != 0.0) {
                done = true;
                break;
            }
        }
        NL_TRY(launch_gmres_update(N, B.ldv, B.V, B.gws, m, jcols, d, st));
        ++*H.launches;
        if (done) break;
    }
    *steps_out = steps;
    return NL_OK;
}

// IR (solver 0: on-the-fly correction; solver 1: the scaled binary16 correction
// of eq. (2.19)) or GMRES-IR (solver 2) for J32 u = b, u0 = 0.
static nl_status linsolve16(int N, const float* J32, int64_t ld32, const __half* LU, int64_t ld16, const TrsvWork& tw,
                            int& epoch, const float* b, float* u, double eta, int maxit, int solver, int m,
                            double gtol, int gcycles, LinBufs& B, Host& H, LinResult* res)
{
    cudaStream_t st = H.st;
    *res = LinResult();
    NL_CUDA_OK(cudaMemsetAsync(u, 0, sizeof(float) * N, st));
    NL_CUDA_OK(cudaMemsetAsync(B.ubest, 0, sizeof(float) * N, st));
    NL_CUDA_OK(cudaMemcpyAsync(B.r, b, sizeof(float) * N, cudaMemcpyDeviceToDevice, st));
    NL_TRY(launch_norm32(N, b, B.partial, B.counter, B.dscal, st));
    ++*H.launches;
    const double nb = H.read(B.dscal);
    double nr = nb, best = nr, prev = nr;
    for (;;) {
        if (nr <= eta * nb) {
            res->converged = 1;
            break;
        }
        if (res->outer >= maxit) break;
        if (solver == 2) {
            int steps = 0;
            NL_TRY(gmres16(N, J32, ld32, LU, ld16, tw, epoch, B.r, B.d, m, gtol, gcycles, B, H, &steps));
            res->iters += steps;
        } else if (solver == 1) {
            // the norm of the current residual: of b before the first correction
            const double* rnorm = res->outer == 0 ? B.dscal : B.dscal + 1;
            NL_TRY(lusolve16h(N, LU, ld16, nullptr, tw.perm, nullptr, B.r, rnorm, nullptr, nullptr, B.d, st));
            ++*H.launches;
            res->iters += 1;
        } else {
            NL_TRY(trsv_solve16(N, LU, ld16, B.r, B.d, tw, ++epoch, st, H.launches));
            res->iters += 1;
        }
        NL_TRY(launch_axpy32(N, 1.0f, B.d, u, st));
        res->outer += 1;
        NL_TRY(launch_gemv_residual(N, J32, ld32, b, u, B.r, B.partial, B.counter, B.dscal + 1, st));
        *H.launches += 2;
        unsigned werr = 0;
        nr = H.read_err(B.dscal + 1, tw.err, &werr);
        if (werr) return NL_ETIMEOUT;  // a triangular solve's bounded wait gave up (reported by the caller)
        if (nr > prev) {
            res->failed = 1;
            NL_CUDA_OK(cudaMemcpyAsync(u, B.ubest, sizeof(float) * N, cudaMemcpyDeviceToDevice, st));
            nr = best;
            break;
        }
        prev = nr;
        if (nr < best) {
            best = nr;
            NL_CUDA_OK(cudaMemcpyAsync(B.ubest, u, sizeof(float) * N, cudaMemcpyDeviceToDevice, st));
        }
    }
    res->relres = nb > 0.0 ? nr / nb : 0.0;
    return NL_OK;
}

}  // namespace nl

using namespace nl;

struct nl_solver {
    int N = 0;
    double c = 0.0;
    nl_config cfg;
    cudaStream_t st = nullptr;
    int64_t ld = 0;  // leading dimension of J32 / J16 / J64 (multiple of 64)
    void* pool = nullptr;
    size_t pool_bytes = 0;
    void* pool64 = nullptr;
    size_t pool64_bytes = 0;
    void* pool32 = nullptr;  // F32 mode and single-precision GMRES-IR factors: the single-precision solve's workspace
    size_t pool32_bytes = 0;
    void* poolc = nullptr;   // single-precision copy of the binary16 factors (gmres_factors32)
    size_t poolc_bytes = 0;
    float* LU32c = nullptr;
    double* pin = nullptr;
    // state
    double *xa = nullptr, *xb = nullptr, *xbest = nullptr, *F = nullptr, *rr = nullptr, *htab = nullptr,
           *partial = nullptr,
           *dscal = nullptr, *gws = nullptr;
    unsigned* counter = nullptr;
    float *J32 = nullptr, *b = nullptr, *u = nullptr;
    float* rs16 = nullptr;  // scale_fp16: power-of-two row factors of J16 = fl16(R J32)
    bool use_fft = false;   // F through the FFT convolution (fft_f)
    FftPlan fft;
    __half* J16 = nullptr;
    int* ipiv = nullptr;
    LinBufs lb;
    LuWork luw;
    bool lookahead = true;  // the binary16 fast path's look-ahead (its side stream lives in luw)
    TrsvWork tw;
    // double-precision mode
    double *J64 = nullptr, *b64 = nullptr, *u64 = nullptr;
    int* ipiv64 = nullptr;
    LuWork luw64;
    TrsvWork tw64;
    TrsvWork tw32;
    int epoch = 0;
    int nb = 128;
    int gemm = 2;
    nl_stats_t stats;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaEvent_t evp[6] = {};  // per-step phase timing (Jacobian, factorisation, linear solve), read once per step
    int tune_count = 0;
    int tune_nb[4] = {0, 0, 0, 0};
    float tune_ms[4] = {0, 0, 0, 0};
};

// Outer block the handle's LU workspace is sized for: the configured one, or
// the largest autotuner candidate.
static int lu_nb_alloc(const nl_config& d) { return d.lu_nb == -1 ? 512 : (d.lu_nb > 0 ? d.lu_nb : 128); }

// Whether F is evaluated through the FFT convolution (nl_config.fft_f).  The
// automatic choice takes it from N = 4096, where its four launches (about
// 45 us) beat the direct sum (61 us at N = 4096, 2.1 ms at N = 32768, GB300).
constexpr int kFftAutoMinN = 4096;
static bool uses_fft(int n, const nl_config& d) { return d.fft_f == 1 || (d.fft_f == 0 && n >= kFftAutoMinN); }

// Device bytes of one handle's main allocation (layout of nl_create).
static size_t solver_bytes(int n, const nl_config& d)
{
    const int m = d.gmres_restart;
    const int nb = lu_nb_alloc(d);
    const int64_t ld = round_up(n, 64), ldv = ld;
    const size_t npart = (size_t)std::max(residual_partials(n), gemv_partials(n)) + 64;
    Carver cv(nullptr);
    cv.take<double>(n);            // xa
    cv.take<double>(n);            // xb
    cv.take<double>(n);            // F
    cv.take<double>(n);            // rr
    cv.take<double>(n);            // xbest
    cv.take<double>(2 * n);        // htab
    cv.take<double>(npart);        // partial
    cv.take<double>(16);           // dscal
    cv.take<unsigned>(4);          // counter
    cv.take<double>(gmres_ws_doubles(m));
    cv.take<float>((size_t)n * ld);     // J32
    cv.take<__half>((size_t)n * ld);    // J16
    cv.take<int>(n);               // ipiv
    cv.take<float>(n);             // rs16
    cv.take<float>(ldv);           // b
    cv.take<float>(ldv);           // u
    for (int q = 0; q < 5; ++q) cv.take<float>(ldv);  // r d t w ubest
    cv.take<float>((size_t)(m + 1) * ldv);            // V
    cv.take<char>(lu_work_bytes(n, nb, false));
    cv.take<char>(trsv_work_bytes(n, false));
    if (uses_fft(n, d)) cv.take<char>(fft_work_bytes(n));
    return cv.off + 256;
}

// Device bytes of the double-precision mode's extra allocation.
static size_t solver64_bytes(int n)
{
    const int64_t ld = round_up(n, 64);
    Carver cv(nullptr);
    cv.take<double>((size_t)n * ld);
    cv.take<double>(n);
    cv.take<double>(n);
    cv.take<int>(n);
    cv.take<char>(lu_work_bytes(n, 64, true));
    cv.take<char>(trsv_work_bytes(n, true));
    return cv.off + 256;
}

// F(x + scale u) (u may be NULL), r and ||F||: direct sum or FFT convolution.
static nl_status eval_F(nl_solver* s, const double* x, const void* u, int u_is_double, double scale, double* xout,
                        double* fnorm_dev, cudaStream_t st)
{
    if (s->use_fft) return launch_residual_fft(s->fft, s->c, x, u, u_is_double, scale, xout, s->F, s->rr, fnorm_dev, st);
    return launch_residual(s->N, s->c, x, u, u_is_double, scale, s->htab, xout, s->F, s->rr, s->partial, s->counter,
                           fnorm_dev, st);
}

// lu_nb = -1: time the factorisation of the Jacobian at x0 = ones for each
// candidate outer block (tcgen05 update where nb is a multiple of 64, SIMT
// otherwise) and keep the fastest.  nb is also the binary16 rounding period.
static nl_status autotune_lu(nl_solver* s)
{
    const int n = s->N;
    // one-level 64 and 128, two-level 256 and 512 (all with the tensor-core update)
    const int cands[4] = {512, 256, 128, 64};
    cudaStream_t st = s->st;
    float* jrs = s->cfg.scale_fp16 ? s->rs16 : nullptr;
    k_fill64<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(n, 1.0, s->xa);
    NL_TRY(eval_F(s, s->xa, nullptr, 0, 0.0, nullptr, s->dscal, st));
    float best = 1e30f;
    int bnb = 128, k = 0;
    for (int nb : cands) {
        if (nb > 128 && 2 * nb > n) continue;  // two levels need at least two outer blocks
        if (nb < 128 && nb > n) continue;
        const int gemm = (nb % 64 == 0 && tc_gemm_supported()) ? 2 : 1;
        float ms_best = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            NL_TRY(launch_jacobian(n, s->c, s->rr, s->htab, s->J32, s->ld, s->J16, s->ld, st, jrs));
            lu_work_carve(s->luw.pnl, n, nb, false, &s->luw);
            if (s->lookahead) NL_TRY(lu_side_prepare(&s->luw, st));
            cudaEventRecord(s->ev[0], st);
            NL_TRY(lu16_factor(n, s->J16, s->ld, s->ipiv, nb, gemm, true, s->luw, st, nullptr));
            cudaEventRecord(s->ev[1], st);
            NL_CUDA_OK(cudaEventSynchronize(s->ev[1]));
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, s->ev[0], s->ev[1]);
            ms_best = std::min(ms_best, ms);
        }
        if (k < 4) {
            s->tune_nb[k] = nb;
            s->tune_ms[k] = ms_best;
            ++k;
        }
        if (ms_best < best) {
            best = ms_best;
            bnb = nb;
        }
    }
    s->tune_count = k;
    s->nb = bnb;
    s->gemm = (bnb % 64 == 0 && tc_gemm_supported()) ? (s->cfg.trailing_gemm ? s->cfg.trailing_gemm : 2) : 1;
    lu_work_carve(s->luw.pnl, n, s->nb, false, &s->luw);
    return NL_OK;
}

static bool valid_mode(int m)
{
    return m == NL_FP64LU || m == NL_IR16 || m == NL_GMRESIR16 || m == NL_IR16_GMRES || m == NL_F32 || m == NL_F16;
}

extern "C" {

nl_status nl_config_default(nl_config* cfg)
{
    if (!cfg) {
        set_error("nl_config_default: cfg is NULL");
        return NL_EINVAL;
    }
    memset(cfg, 0, sizeof(*cfg));
    cfg->eta_j = 1e-4;
    cfg->ir_maxit = 20;
    cfg->gmres_restart = 30;
    cfg->gmres_tol = 1e-4;
    cfg->gmres_maxcycles = 10;
    cfg->newton_maxit = 30;
    cfg->tau_a = 0.0;
    cfg->lu_nb = 0;
    cfg->trailing_gemm = 0;
    return NL_OK;
}

const char* nl_last_error(void) { return get_error(); }

nl_status nl_kernel_timing(const char* kernel_class, int* launches, double* total_ms)
{
    std::lock_guard<std::mutex> lock(g_kt.mu);
    double tot = 0.0;
    int n = 0;
    for (auto& p : g_kt.ev) {
        float ms = 0.0f;
        if (cudaEventSynchronize(p.second) == cudaSuccess && cudaEventElapsedTime(&ms, p.first, p.second) == cudaSuccess) {
            tot += ms;
            ++n;
        }
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
    }
    g_kt.ev.clear();
    g_kt.open = -1;
    if (launches) *launches = n;
    if (total_ms) *total_ms = tot;
    g_kt.cls = kernel_class ? kernel_class : "";
    return NL_OK;
}
const char* nl_version(void) { return "newton3p-gb300 0.2 (sm_103a)"; }

nl_status nl_debug_fail_allocs(int count)
{
    if (count < 0) {
        set_error("nl_debug_fail_allocs: count < 0");
        return NL_EINVAL;
    }
    g_fail_allocs.store(count);
    return NL_OK;
}

nl_status nl_create(int64_t N, double c, const nl_config* cfg, nl_solver** out)
{
    set_error("");
    if (!out || N < 1 || N > 32768 || !(c >= 0.0 && c < 1.0)) {
        set_error("nl_create: need N in [1, 32768], 0 <= c < 1 and out != NULL");
        return NL_EINVAL;
    }
    nl_config d;
    nl_config_default(&d);
    if (cfg) d = *cfg;
    if (d.gmres_restart < 1 || d.gmres_restart > 62 || d.ir_maxit < 0 || d.newton_maxit < 0 || d.lu_path < 0 ||
        d.lu_path > 1 || !(d.trsv_cluster == -1 || d.trsv_cluster == 0 || d.trsv_cluster == 4 ||
                           d.trsv_cluster == 8 || d.trsv_cluster == 16) ||
        !(d.lu_stream == 0 || d.lu_stream == -1 || d.lu_stream == 256) || d.ir_variant < 0 || d.ir_variant > 1 ||
        d.gmres_factors32 < 0 || d.gmres_factors32 > 1 || d.lu16_arith < 0 || d.lu16_arith > 1 ||
        d.newton_maxit >= NL_MAX_HIST || (d.lu_nb > 0 && !lu16_nb_valid(d.lu_nb)) ||
        d.lu_nb < -1 || d.scale_fp16 < 0 || d.scale_fp16 > 1 || d.fft_f < -1 || d.fft_f > 1 ||
        d.trailing_gemm < 0 || d.trailing_gemm > 2 || d.lu_lookahead < -1 || d.lu_lookahead > 0 ||
        (d.scale_fp16 && (d.ir_variant || d.gmres_factors32 || d.lu16_arith))) {
        set_error("nl_create: invalid configuration");
        return NL_EINVAL;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        set_error("nl_create: no CUDA device");
        return NL_ECUDA;
    }
    nl_solver* s = new nl_solver();
    s->N = (int)N;
    s->c = c;
    s->cfg = d;
    s->nb = d.lu_nb > 0 ? d.lu_nb : 128;  // the autotuner (lu_nb = -1) may change it; buffers fit lu_nb_alloc
    s->gemm = d.trailing_gemm ? d.trailing_gemm : 2;
    if (s->gemm == 2 && (!tc_gemm_supported() || s->nb % 64)) s->gemm = 1;
    s->ld = round_up(N, 64);
    const int n = s->N;
    const int m = d.gmres_restart;
    const int64_t ldv = round_up(N, 64);
    const size_t npart = (size_t)std::max(residual_partials(n), gemv_partials(n)) + 64;
    const size_t bytes = solver_bytes(n, d);
    if (dev_malloc(&s->pool, bytes) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        set_error("nl_create: cudaMalloc of %zu bytes failed", bytes);
        return NL_ENOMEM;
    }
    s->pool_bytes = bytes;
    cudaMemset(s->pool, 0, bytes);
    Carver cv(s->pool);
    s->xa = cv.take<double>(n);
    s->xb = cv.take<double>(n);
    s->F = cv.take<double>(n);
    s->rr = cv.take<double>(n);
    s->xbest = cv.take<double>(n);
    s->htab = cv.take<double>(2 * n);
    s->partial = cv.take<double>(npart);
    s->dscal = cv.take<double>(16);
    s->counter = cv.take<unsigned>(4);
    s->gws = cv.take<double>(gmres_ws_doubles(m));
    s->J32 = cv.take<float>((size_t)n * s->ld);
    s->J16 = cv.take<__half>((size_t)n * s->ld);
    s->ipiv = cv.take<int>(n);
    s->rs16 = cv.take<float>(n);
    s->b = cv.take<float>(ldv);
    s->u = cv.take<float>(ldv);
    s->lb.r = cv.take<float>(ldv);
    s->lb.d = cv.take<float>(ldv);
    s->lb.t = cv.take<float>(ldv);
    s->lb.w = cv.take<float>(ldv);
    s->lb.ubest = cv.take<float>(ldv);
    s->lb.V = cv.take<float>((size_t)(m + 1) * ldv);
    s->lb.ldv = ldv;
    s->lb.gws = s->gws;
    s->lb.partial = s->partial;
    s->lb.counter = s->counter;
    s->lb.dscal = s->dscal + 4;
    lu_work_carve(cv.take<char>(lu_work_bytes(n, lu_nb_alloc(d), false)), n, s->nb, false, &s->luw);
    trsv_work_carve(cv.take<char>(trsv_work_bytes(n, false)), n, false, &s->tw);
    s->use_fft = uses_fft(n, d);
    if (s->use_fft) fft_work_carve(cv.take<char>(fft_work_bytes(n)), n, &s->fft);
    s->tw.cluster = d.trsv_cluster;
    s->tw.wait_limit = d.wait_limit;
    s->tw.rs = d.scale_fp16 ? s->rs16 : nullptr;
    s->luw.stream = d.lu_stream;
    s->lookahead = d.lu_lookahead == 0;
    bool evs_ok = true;
    for (auto& e : s->evp) evs_ok = evs_ok && cudaEventCreate(&e) == cudaSuccess;
    if (!evs_ok || cudaMallocHost((void**)&s->pin, 64) != cudaSuccess || cudaEventCreate(&s->ev[0]) != cudaSuccess ||
        cudaEventCreate(&s->ev[1]) != cudaSuccess) {
        cudaFree(s->pool);
        delete s;
        set_error("nl_create: host/event allocation failed");
        return NL_ENOMEM;
    }
    if (launch_htab(n, s->htab, s->st) != NL_OK || (s->use_fft && fft_prepare(s->fft, s->st) != NL_OK) ||
        cudaStreamSynchronize(s->st) != cudaSuccess) {
        nl_destroy(s);
        return NL_ECUDA;
    }
    memset(&s->stats, 0, sizeof(s->stats));
    if (d.lu_nb < 0) {
        nl_status ts = autotune_lu(s);
        if (ts != NL_OK) {
            nl_destroy(s);
            return ts;
        }
    }
    *out = s;
    return NL_OK;
}

nl_status nl_set_stream(nl_solver* s, void* stream)
{
    if (!s) {
        set_error("nl_set_stream: NULL handle");
        return NL_EINVAL;
    }
    s->st = (cudaStream_t)stream;
    return NL_OK;
}

int64_t nl_device_bytes(const nl_solver* s)
{
    return s ? (int64_t)(s->pool_bytes + s->pool64_bytes + s->pool32_bytes + s->poolc_bytes) : 0;
}

int64_t nl_footprint_bytes(int64_t N, nl_mode mode, const nl_config* cfg)
{
    if (N < 1 || N > 32768 || !valid_mode(mode)) return -1;
    nl_config d;
    nl_config_default(&d);
    if (cfg) d = *cfg;
    size_t b = solver_bytes((int)N, d);
    if (mode == NL_FP64LU) b += solver64_bytes((int)N);
    const bool f32fac = d.gmres_factors32 && (mode == NL_GMRESIR16 || mode == NL_IR16_GMRES);
    if (mode == NL_F32 || f32fac) b += trsv_work_bytes((int)N, true) + 256;
    if (f32fac) b += (size_t)N * round_up((int)N, 64) * sizeof(float) + 256;
    return (int64_t)b;
}

nl_status nl_set_c(nl_solver* s, double c)
{
    if (!s || !(c >= 0.0 && c < 1.0)) {
        set_error("nl_set_c: need a handle and 0 <= c < 1");
        return NL_EINVAL;
    }
    s->c = c;
    return NL_OK;
}

void nl_destroy(nl_solver* s)
{
    if (!s) return;
    if (s->st) cudaStreamSynchronize(s->st);
    else cudaDeviceSynchronize();
    lu_side_release(&s->luw);
    if (s->pool) cudaFree(s->pool);
    if (s->pool64) cudaFree(s->pool64);
    if (s->pool32) cudaFree(s->pool32);
    if (s->poolc) cudaFree(s->poolc);
    if (s->pin) cudaFreeHost(s->pin);
    if (s->ev[0]) cudaEventDestroy(s->ev[0]);
    if (s->ev[1]) cudaEventDestroy(s->ev[1]);
    for (auto& e : s->evp)
        if (e) cudaEventDestroy(e);
    delete s;
}

static nl_status ensure_fp64(nl_solver* s)
{
    if (s->pool64) return NL_OK;
    const int n = s->N;
    const int nb64 = 64;
    const size_t bytes = solver64_bytes(n);
    if (dev_malloc(&s->pool64, bytes) != cudaSuccess) {
        cudaGetLastError();
        s->pool64 = nullptr;
        set_error("double-precision Jacobian: cudaMalloc of %zu bytes failed", bytes);
        return NL_ENOMEM;
    }
    s->pool64_bytes = bytes;
    cudaMemsetAsync(s->pool64, 0, bytes, s->st);
    Carver cv(s->pool64);
    s->J64 = cv.take<double>((size_t)n * s->ld);
    s->b64 = cv.take<double>(n);
    s->u64 = cv.take<double>(n);
    s->ipiv64 = cv.take<int>(n);
    lu_work_carve(cv.take<char>(lu_work_bytes(n, nb64, true)), n, nb64, true, &s->luw64);
    trsv_work_carve(cv.take<char>(trsv_work_bytes(n, true)), n, true, &s->tw64);
    return NL_OK;
}

// F32 mode: the blocked single-precision solve uses the double layout of its
// workspace (64-row blocks).
static nl_status ensure_fp32(nl_solver* s)
{
    if (s->pool32) return NL_OK;
    const size_t bytes = trsv_work_bytes(s->N, true);
    if (dev_malloc(&s->pool32, bytes) != cudaSuccess) {
        cudaGetLastError();
        s->pool32 = nullptr;
        set_error("single-precision solve: cudaMalloc of %zu bytes failed", bytes);
        return NL_ENOMEM;
    }
    s->pool32_bytes = bytes;
    cudaMemsetAsync(s->pool32, 0, bytes, s->st);
    trsv_work_carve(s->pool32, s->N, true, &s->tw32);
    return NL_OK;
}

// gmres_factors32: the single-precision copy of the binary16 factors.
static nl_status ensure_factors32(nl_solver* s)
{
    NL_TRY(ensure_fp32(s));
    if (s->poolc) return NL_OK;
    const size_t bytes = (size_t)s->N * s->ld * sizeof(float);
    if (dev_malloc(&s->poolc, bytes) != cudaSuccess) {
        cudaGetLastError();
        s->poolc = nullptr;
        set_error("single-precision factor copy: cudaMalloc of %zu bytes failed", bytes);
        return NL_ENOMEM;
    }
    s->poolc_bytes = bytes;
    s->LU32c = (float*)s->poolc;
    return NL_OK;
}

static float elapsed_ms(nl_solver* s)
{
    float ms = 0.0f;
    cudaEventSynchronize(s->ev[1]);
    cudaEventElapsedTime(&ms, s->ev[0], s->ev[1]);
    return ms;
}

static float pair_ms(cudaEvent_t a, cudaEvent_t b)
{
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        cudaGetLastError();
        ms = 0.0f;
    }
    return ms;
}

// Clears the handle's device error words (after a bounded wait gave up), so
// that the next solve starts clean.
static void clear_error_words(nl_solver* s)
{
    unsigned* tce = tc_error_word();
    cudaMemsetAsync(s->tw.err, 0, sizeof(unsigned), s->st);
    if (s->tw64.err) cudaMemsetAsync(s->tw64.err, 0, sizeof(unsigned), s->st);
    if (s->tw32.err) cudaMemsetAsync(s->tw32.err, 0, sizeof(unsigned), s->st);
    if (tce) cudaMemsetAsync(tce, 0, sizeof(unsigned), s->st);
    cudaStreamSynchronize(s->st);
}

// The residual norm of the new iterate and the device error words in one
// round trip; an error word set by a bounded wait that gave up is cleared and
// reported as NL_ETIMEOUT.
static nl_status read_step_end(nl_solver* s, const double* fn_dev, double* fn)
{
    char* p = reinterpret_cast<char*>(s->pin);
    unsigned* tce = tc_error_word();
    NL_CUDA_OK(cudaMemcpyAsync(p, fn_dev, sizeof(double), cudaMemcpyDeviceToHost, s->st));
    memset(p + 8, 0, 16);
    NL_CUDA_OK(cudaMemcpyAsync(p + 8, s->tw.err, sizeof(unsigned), cudaMemcpyDeviceToHost, s->st));
    if (s->tw64.err) NL_CUDA_OK(cudaMemcpyAsync(p + 12, s->tw64.err, sizeof(unsigned), cudaMemcpyDeviceToHost, s->st));
    if (tce) NL_CUDA_OK(cudaMemcpyAsync(p + 16, tce, sizeof(unsigned), cudaMemcpyDeviceToHost, s->st));
    if (s->tw32.err) NL_CUDA_OK(cudaMemcpyAsync(p + 20, s->tw32.err, sizeof(unsigned), cudaMemcpyDeviceToHost, s->st));
    NL_CUDA_OK(cudaStreamSynchronize(s->st));
    memcpy(fn, p, sizeof(double));
    unsigned e[4];
    memcpy(e, p + 8, sizeof(e));
    if (e[0] | e[1] | e[2] | e[3]) {
        set_error("a device-side bounded wait gave up (error word 0x%x/0x%x/0x%x/0x%x)", e[0], e[1], e[2], e[3]);
        clear_error_words(s);
        return NL_ETIMEOUT;
    }
    return NL_OK;
}

static nl_status solve_impl(nl_solver* s, const double* x0, bool x0_host, double tol, nl_mode mode, double* x_out,
                            bool out_host)
{
    auto t_start = std::chrono::steady_clock::now();
    const int n = s->N;
    cudaStream_t st = s->st;
    nl_stats_t& S = s->stats;
    memset(&S, 0, sizeof(S));
    S.mode = mode;
    S.lu_nb = (mode == NL_FP64LU) ? 64 : s->nb;
    S.lu_tune_count = s->tune_count;
    for (int k = 0; k < 4; ++k) {
        S.lu_tune_nb[k] = s->tune_nb[k];
        S.lu_tune_ms[k] = s->tune_ms[k];
    }
    int launches = 0;
    Host H{s->pin, st, &launches};
    if (mode == NL_F16 && s->cfg.scale_fp16) {
        set_error("nl_solve: scale_fp16 applies to the three-precision modes, not NL_F16");
        return NL_EINVAL;
    }
    float* jrs = s->cfg.scale_fp16 ? s->rs16 : nullptr;
    if (mode == NL_FP64LU) NL_TRY(ensure_fp64(s));
    if (mode == NL_F32) NL_TRY(ensure_fp32(s));
    const bool f32fac = s->cfg.gmres_factors32 && (mode == NL_GMRESIR16 || mode == NL_IR16_GMRES);
    if (f32fac) NL_TRY(ensure_factors32(s));
    s->lb.LU32 = f32fac ? s->LU32c : nullptr;
    s->lb.tw32 = f32fac ? &s->tw32 : nullptr;

    double* x = s->xa;
    double* xn = s->xb;
    if (x0) {
        NL_CUDA_OK(cudaMemcpyAsync(x, x0, sizeof(double) * n, x0_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                   st));
    } else {
        k_fill64<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(n, 1.0, x);
        ++launches;
    }
    double* fn_dev = s->dscal;
    cudaEventRecord(s->ev[0], st);
    NL_TRY(eval_F(s, x, nullptr, 0, 0.0, nullptr, fn_dev, st));
    cudaEventRecord(s->ev[1], st);
    ++launches;
    const double f0 = H.read(fn_dev);
    S.t_f_ms += elapsed_ms(s);
    double fn = f0;
    const double tau = tol * f0 + s->cfg.tau_a;
    S.fnorm0 = f0;
    S.hist[0] = 1.0;
    int it = 0;
    bool gm_sticky = false;  // NL_IR16_GMRES: GMRES-IR from the first stalled step on
    nl_status status = NL_ENOTCONV;
    // The iterate with the smallest ||F|| so far (returned unless the solve
    // converges): its step index, its norm, and whether it has been copied to
    // xbest (it is, as soon as a later step fails to improve on it, while it
    // still sits in the other iterate buffer).
    int best_it = 0;
    double best_fn = f0;
    bool best_saved = false;
    while (!(fn <= tau)) {
        if (!std::isfinite(fn)) {
            status = NL_ENUMERIC;
            set_error("non-finite residual norm");
            break;
        }
        if (it >= s->cfg.newton_maxit) break;
        // Jacobian (the phases' times are read after the step's one synchronisation)
        cudaEventRecord(s->evp[0], st);
        if (mode == NL_FP64LU)
            NL_TRY(launch_jacobian64(n, s->c, s->rr, s->htab, s->J64, s->ld, st));
        else
            NL_TRY(launch_jacobian(n, s->c, s->rr, s->htab, s->J32, s->ld, s->J16, s->ld, st, jrs));
        cudaEventRecord(s->evp[1], st);
        ++launches;
        // factorisation
        cudaEventRecord(s->evp[2], st);
        int info = 0, iflag[2] = {0, 0};
        const bool pivoted_only = s->cfg.lu_path == 1;
        if (mode == NL_FP64LU) {
            NL_TRY(lu64_factor(n, s->J64, s->ld, s->ipiv64, 64, !pivoted_only, s->luw64, st, &launches));
            NL_CUDA_OK(cudaMemcpyAsync(s->pin, s->luw64.info, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
            NL_CUDA_OK(cudaStreamSynchronize(st));
            memcpy(iflag, s->pin, sizeof(iflag));
            if (iflag[1]) {  // interchanges needed: re-form J and factor with them
                NL_TRY(launch_jacobian64(n, s->c, s->rr, s->htab, s->J64, s->ld, st));
                NL_TRY(lu64_factor(n, s->J64, s->ld, s->ipiv64, 64, false, s->luw64, st, &launches));
                NL_CUDA_OK(cudaMemcpyAsync(s->pin, s->luw64.info, sizeof(int), cudaMemcpyDeviceToHost, st));
                ++launches;
                ++S.lu_pivoted;
            }
            NL_TRY(trsv_prepare64(n, s->J64, s->ld, s->ipiv64, s->tw64, st, &launches));
        } else if (s->cfg.lu16_arith && mode != NL_F32) {
            // every operation of the factorisation rounded to binary16 (interchanges included)
            NL_TRY(lu16_factor_arith(n, s->J16, s->ld, s->ipiv, s->luw, st));
            ++launches;
            NL_CUDA_OK(cudaMemcpyAsync(s->pin, s->luw.info, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
            if (mode != NL_F16) NL_TRY(trsv_prepare16(n, s->J16, s->ld, s->ipiv, s->tw, st, &launches));
            if (f32fac) {
                NL_TRY(launch_promote16(n, s->J16, s->ld, s->LU32c, s->ld, st));
                NL_TRY(trsv_prepare32(n, s->LU32c, s->ld, s->ipiv, s->tw32, st, &launches));
                ++launches;
            }
            NL_CUDA_OK(cudaStreamSynchronize(st));
            memcpy(iflag, s->pin, sizeof(iflag));
            if (iflag[1]) {
                status = NL_ENUMERIC;
                set_error("binary16 overflow in the factorisation");
                break;
            }
        } else if (mode == NL_F32) {
            // two-precision Newton, F32: J32 factored in place in single precision
            NL_TRY(lu32_factor(n, s->J32, s->ld, s->ipiv, std::min(s->nb, 128), s->luw, st, &launches));
            NL_CUDA_OK(cudaMemcpyAsync(s->pin, s->luw.info, sizeof(int), cudaMemcpyDeviceToHost, st));
            NL_TRY(trsv_prepare32(n, s->J32, s->ld, s->ipiv, s->tw32, st, &launches));
        } else {
            // the fast path's outcome is read once, after the triangular solves' set-up
            // has been queued behind it (redone below in the rare case of interchanges)
            if (s->lookahead && !pivoted_only) NL_TRY(lu_side_prepare(&s->luw, st));
            NL_TRY(lu16_factor(n, s->J16, s->ld, s->ipiv, s->nb, s->gemm, !pivoted_only, s->luw, st, &launches));
            NL_CUDA_OK(cudaMemcpyAsync(s->pin, s->luw.info, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
            if (mode != NL_F16) NL_TRY(trsv_prepare16(n, s->J16, s->ld, s->ipiv, s->tw, st, &launches));
            NL_CUDA_OK(cudaStreamSynchronize(st));
            memcpy(iflag, s->pin, sizeof(iflag));
            if (iflag[1]) {
                NL_TRY(launch_jacobian(n, s->c, s->rr, s->htab, s->J32, s->ld, s->J16, s->ld, st, jrs));
                NL_TRY(lu16_factor(n, s->J16, s->ld, s->ipiv, s->nb, s->gemm, false, s->luw, st, &launches));
                NL_CUDA_OK(cudaMemcpyAsync(s->pin, s->luw.info, sizeof(int), cudaMemcpyDeviceToHost, st));
                ++launches;
                ++S.lu_pivoted;
                if (mode != NL_F16) NL_TRY(trsv_prepare16(n, s->J16, s->ld, s->ipiv, s->tw, st, &launches));
            }
            if (f32fac) {
                NL_TRY(launch_promote16(n, s->J16, s->ld, s->LU32c, s->ld, st));
                NL_TRY(trsv_prepare32(n, s->LU32c, s->ld, s->ipiv, s->tw32, st, &launches));
                ++launches;
            }
        }
        cudaEventRecord(s->evp[3], st);
        NL_CUDA_OK(cudaStreamSynchronize(st));
        memcpy(&info, s->pin, sizeof(int));
        if (info != 0) {
            status = NL_ESINGULAR;
            set_error("zero pivot at column %d", info);
            break;
        }
        // linear solve for the scaled step
        cudaEventRecord(s->evp[4], st);
        const void* ustep;
        int u_is_double = 0;
        if (mode == NL_FP64LU) {
            NL_TRY(launch_scale_rhs64(n, s->F, fn_dev, s->b64, st));
            NL_TRY(trsv_solve64(n, s->J64, s->ld, s->b64, s->u64, s->tw64, ++s->epoch, st, &launches));
            ++launches;
            ustep = s->u64;
            u_is_double = 1;
        } else if (mode == NL_F32) {
            // one single-precision solve with the single-precision factors
            NL_TRY(launch_scale_rhs32(n, s->F, fn_dev, s->b, st));
            NL_TRY(trsv_solve32(n, s->J32, s->ld, s->b, s->u, s->tw32, ++s->epoch, st, &launches));
            ++launches;
            ustep = s->u;
        } else if (mode == NL_F16) {
            // one binary16-arithmetic solve of fl16(-F/||F||) with the binary16 factors
            NL_TRY(lusolve16h(n, s->J16, s->ld, s->ipiv, nullptr, s->F, nullptr, fn_dev, nullptr, nullptr, s->u, st));
            ++launches;
            ustep = s->u;
        } else {
            NL_TRY(launch_scale_rhs32(n, s->F, fn_dev, s->b, st));
            ++launches;
            LinResult lr;
            nl_status ls = linsolve16(n, s->J32, s->ld, s->J16, s->ld, s->tw, s->epoch, s->b, s->u, s->cfg.eta_j,
                                      s->cfg.ir_maxit, (mode == NL_GMRESIR16 || gm_sticky) ? 2 : s->cfg.ir_variant,
                                      s->cfg.gmres_restart, s->cfg.gmres_tol, s->cfg.gmres_maxcycles, s->lb, H, &lr);
            if (ls == NL_ETIMEOUT) {  // a triangular solve gave up: no step from this factorisation
                clear_error_words(s);
                set_error("a device-side bounded wait gave up (triangular solve)");
                status = NL_ETIMEOUT;
                break;
            }
            NL_TRY(ls);
            if (mode == NL_IR16_GMRES && !gm_sticky && !lr.converged) {
                // IR stalled: redo this step with GMRES-IR, and keep it for the rest of the solve
                gm_sticky = true;
                LinResult lg;
                ls = linsolve16(n, s->J32, s->ld, s->J16, s->ld, s->tw, s->epoch, s->b, s->u, s->cfg.eta_j,
                                s->cfg.ir_maxit, 2, s->cfg.gmres_restart, s->cfg.gmres_tol, s->cfg.gmres_maxcycles,
                                s->lb, H, &lg);
                if (ls == NL_ETIMEOUT) {
                    clear_error_words(s);
                    set_error("a device-side bounded wait gave up (triangular solve)");
                    status = NL_ETIMEOUT;
                    break;
                }
                NL_TRY(ls);
                lg.iters += lr.iters;
                lg.outer += lr.outer;
                lg.failed = 1;
                lr = lg;
            }
            S.lin_iters[it] = lr.iters;
            S.lin_outer[it] = lr.outer;
            S.lin_failed[it] = lr.failed;
            S.lin_relres[it] = lr.relres;
            ustep = s->u;
        }
        cudaEventRecord(s->evp[5], st);
        // x_{n+1} = x_n + ||F|| u, fused with F(x_{n+1}); its norm and the device error
        // words come back with the step's one synchronisation
        NL_TRY(eval_F(s, x, ustep, u_is_double, fn, xn, fn_dev, st));
        ++launches;
        nl_status e = read_step_end(s, fn_dev, &fn);
        S.t_jac_ms += pair_ms(s->evp[0], s->evp[1]);
        S.t_lu_ms += pair_ms(s->evp[2], s->evp[3]);
        S.t_lin_ms += pair_ms(s->evp[4], s->evp[5]);
        std::swap(x, xn);
        ++it;
        S.hist[it] = f0 > 0.0 ? fn / f0 : 0.0;
        if (e != NL_OK) {  // a bounded wait gave up: this step's iterate is not trusted
            status = e;
            break;
        }
        if (fn < best_fn) {
            best_it = it;
            best_fn = fn;
            best_saved = false;
        } else if (best_it == it - 1 && !best_saved) {
            NL_CUDA_OK(cudaMemcpyAsync(s->xbest, xn, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
            best_saved = true;
        }
    }
    if (status != NL_ETIMEOUT && fn <= tau) status = NL_OK;
    // NL_OK: the final iterate; otherwise the best one seen (the final one when it is the best)
    const double* xres = x;
    double fres = fn;
    if (status != NL_OK && best_it != it) {
        if (best_it == it - 1 && !best_saved) xres = xn;
        else xres = s->xbest;
        fres = best_fn;
    }
    NL_CUDA_OK(cudaMemcpyAsync(x_out, xres, sizeof(double) * n,
                               out_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    NL_CUDA_OK(cudaStreamSynchronize(st));
    S.status = status;
    S.newton_iters = it;
    S.fnorm = fres;
    S.gpu_launches = launches;
    S.t_total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    return status;
}

nl_status nl_solve(nl_solver* s, const double* x0, double tol, nl_mode mode, double* x_out)
{
    set_error("");
    if (!s || !x_out || !valid_mode(mode) || !(tol >= 0.0)) {
        set_error("nl_solve: bad argument");
        return NL_EINVAL;
    }
    return solve_impl(s, x0, true, tol, mode, x_out, true);
}

nl_status nl_solve_device(nl_solver* s, const double* x0_dev, double tol, nl_mode mode, double* x_out_dev)
{
    set_error("");
    if (!s || !x_out_dev || !valid_mode(mode) || !(tol >= 0.0)) {
        set_error("nl_solve_device: bad argument");
        return NL_EINVAL;
    }
    return solve_impl(s, x0_dev, false, tol, mode, x_out_dev, false);
}

nl_status nl_stats(const nl_solver* s, nl_stats_t* out)
{
    if (!s || !out) {
        set_error("nl_stats: NULL argument");
        return NL_EINVAL;
    }
    *out = s->stats;
    return NL_OK;
}

// ------------------------------------------------------ kernel-level API --

nl_status nl_k_residual(int64_t N, double c, const double* x, const void* u, int u_is_double, double fnorm_scale,
                        double* x_out, double* F, double* r, double* fnorm_dev, void* stream)
{
    if (N < 1 || N > 32768 || !x || !F || !r || !fnorm_dev || (u && !x_out) || (x_out && x_out == x)) {
        set_error("nl_k_residual: bad argument");
        return NL_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int n = (int)N;
    double *htab = nullptr, *partial = nullptr;
    unsigned* counter = nullptr;
    const size_t np = residual_partials(n);
    NL_CUDA_OK(cudaMallocAsync((void**)&htab, sizeof(double) * (2 * n + np) + 256, st));
    partial = htab + 2 * n;
    counter = (unsigned*)(partial + np);
    NL_CUDA_OK(cudaMemsetAsync(counter, 0, sizeof(unsigned), st));
    nl_status s = launch_htab(n, htab, st);
    if (s == NL_OK)
        s = launch_residual(n, c, x, u, u_is_double, fnorm_scale, htab, x_out, F, r, partial, counter, fnorm_dev, st);
    cudaFreeAsync(htab, st);
    return s;
}

nl_status nl_k_residual_fft(int64_t N, double c, const double* x, const void* u, int u_is_double,
                            double fnorm_scale, double* x_out, double* F, double* r, double* fnorm_dev, void* stream)
{
    if (N < 1 || N > 32768 || !x || !F || !r || !fnorm_dev || (u && !x_out) || (x_out && x_out == x)) {
        set_error("nl_k_residual_fft: bad argument");
        return NL_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int n = (int)N;
    void* wk = nullptr;
    NL_CUDA_OK(cudaMallocAsync(&wk, fft_work_bytes(n), st));
    FftPlan p;
    fft_work_carve(wk, n, &p);
    nl_status s = fft_prepare(p, st);
    if (s == NL_OK) s = launch_residual_fft(p, c, x, u, u_is_double, fnorm_scale, x_out, F, r, fnorm_dev, st);
    cudaFreeAsync(wk, st);
    return s;
}

static nl_status jacobian_entry(int64_t N, double c, const double* r, float* J32, int64_t ld32, void* J16,
                                int64_t ld16, float* rs, void* stream, const char* name)
{
    if (N < 1 || N > 32768 || !r || (J32 && ld32 < N) || (J16 && ld16 < N)) {
        set_error("%s: bad argument", name);
        return NL_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int n = (int)N;
    double* htab = nullptr;
    NL_CUDA_OK(cudaMallocAsync((void**)&htab, sizeof(double) * 2 * n, st));
    nl_status s = launch_htab(n, htab, st);
    if (s == NL_OK) s = launch_jacobian(n, c, r, htab, J32, ld32, (__half*)J16, ld16, st, rs);
    cudaFreeAsync(htab, st);
    return s;
}

nl_status nl_k_jacobian(int64_t N, double c, const double* r, float* J32, int64_t ld32, void* J16, int64_t ld16,
                        void* stream)
{
    return jacobian_entry(N, c, r, J32, ld32, J16, ld16, nullptr, stream, "nl_k_jacobian");
}

nl_status nl_k_jacobian_scaled(int64_t N, double c, const double* r, float* J32, int64_t ld32, void* J16,
                               int64_t ld16, float* rs, void* stream)
{
    if (!rs) {
        set_error("nl_k_jacobian_scaled: rs is NULL");
        return NL_EINVAL;
    }
    return jacobian_entry(N, c, r, J32, ld32, J16, ld16, rs, stream, "nl_k_jacobian_scaled");
}

nl_status nl_k_jacobian64(int64_t N, double c, const double* r, double* J64, int64_t ld, void* stream)
{
    if (N < 1 || N > 32768 || !r || !J64 || ld < N) {
        set_error("nl_k_jacobian64: bad argument");
        return NL_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int n = (int)N;
    double* htab = nullptr;
    NL_CUDA_OK(cudaMallocAsync((void**)&htab, sizeof(double) * 2 * n, st));
    nl_status s = launch_htab(n, htab, st);
    if (s == NL_OK) s = launch_jacobian64(n, c, r, htab, J64, ld, st);
    cudaFreeAsync(htab, st);
    return s;
}

}  // extern "C"

// Factor with the no-interchange fast path, falling back to the interchanging
// path (from a saved copy of A) when partial pivoting would swap rows.
template <typename S>
static nl_status lu_entry(int64_t N, S* A, int64_t ld, int32_t* ipiv, int nb, int gemm, int path, int32_t* info_host,
                          cudaStream_t st, bool fp64)
{
    const int n = (int)N;
    const size_t lw = lu_work_bytes(n, nb, fp64);
    const size_t copy = (path == 1) ? 0 : (size_t)n * ld * sizeof(S);
    void* wk = nullptr;
    NL_CUDA_OK(cudaMallocAsync(&wk, lw + copy + 256, st));
    LuWork w;
    lu_work_carve(wk, n, nb, fp64, &w);
    if (path == 2) {  // the fast path with two launches per panel (no streaming panel)
        w.stream = -1;
        path = 0;
    }
    struct SideGuard {
        LuWork* w;
        ~SideGuard() { lu_side_release(w); }
    } side_guard{&w};
    if (path == 4) {  // the fast path with look-ahead (a side stream for the trailing updates)
        const nl_status ps = lu_side_prepare(&w, st);
        if (ps != NL_OK) {
            cudaFreeAsync(wk, st);
            return ps;
        }
        path = 0;
    }
    S* backup = (S*)((char*)wk + round_up(lw, 256));
    int iflag[2] = {0, 0};
    nl_status s = NL_OK;
    if (path != 1) {
        NL_CUDA_OK(cudaMemcpyAsync(backup, A, copy, cudaMemcpyDeviceToDevice, st));
        if constexpr (std::is_same<S, __half>::value)
            s = lu16_factor(n, A, ld, ipiv, nb, gemm, true, w, st, nullptr);
        else
            s = lu64_factor(n, A, ld, ipiv, nb, true, w, st, nullptr);
        if (s == NL_OK && cudaMemcpyAsync(iflag, w.info, 2 * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            s = NL_ECUDA;
        if (s == NL_OK && cudaStreamSynchronize(st) != cudaSuccess) s = NL_ECUDA;
    }
    if (s == NL_OK && (path == 1 || iflag[1])) {
        if (path != 1) NL_CUDA_OK(cudaMemcpyAsync(A, backup, copy, cudaMemcpyDeviceToDevice, st));
        if constexpr (std::is_same<S, __half>::value)
            s = lu16_factor(n, A, ld, ipiv, nb, gemm, false, w, st, nullptr);
        else
            s = lu64_factor(n, A, ld, ipiv, nb, false, w, st, nullptr);
        if (s == NL_OK && cudaMemcpyAsync(iflag, w.info, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            s = NL_ECUDA;
    }
    cudaFreeAsync(wk, st);
    NL_CUDA_OK(cudaStreamSynchronize(st));
    unsigned* tce = tc_error_word();
    if (s == NL_OK && tce) {
        unsigned e = 0;
        NL_CUDA_OK(cudaMemcpy(&e, tce, sizeof(unsigned), cudaMemcpyDeviceToHost));
        if (e) {
            cudaMemset(tce, 0, sizeof(unsigned));
            set_error("tensor-core update: bounded wait gave up");
            return NL_ETIMEOUT;
        }
    }
    if (info_host) *info_host = iflag[0];
    if (s == NL_OK && iflag[0]) return NL_ESINGULAR;
    return s;
}

// nl_lu16 path 3: the binary16-arithmetic factorisation.
static nl_status lu16_arith_entry(int n, __half* A, int64_t ld, int32_t* ipiv, int32_t* info_host, cudaStream_t st)
{
    void* wk = nullptr;
    NL_CUDA_OK(cudaMallocAsync(&wk, lu_work_bytes(n, 128, false) + 256, st));
    LuWork w;
    lu_work_carve(wk, n, 128, false, &w);
    int iflag[2] = {0, 0};
    nl_status s = lu16_factor_arith(n, A, ld, ipiv, w, st);
    if (s == NL_OK && cudaMemcpyAsync(iflag, w.info, 2 * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        s = NL_ECUDA;
    unsigned e = 0;
    unsigned* tce = tc_error_word();
    unsigned* err = tce ? tce : (unsigned*)(w.info + 2);
    if (s == NL_OK && cudaMemcpyAsync(&e, err, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        s = NL_ECUDA;
    cudaFreeAsync(wk, st);
    NL_CUDA_OK(cudaStreamSynchronize(st));
    if (s != NL_OK) return s;
    if (e) {
        if (tce) cudaMemset(tce, 0, sizeof(unsigned));
        set_error("binary16-arithmetic LU: a grid barrier gave up");
        return NL_ETIMEOUT;
    }
    if (info_host) *info_host = iflag[1] ? -1 : iflag[0];
    if (iflag[1]) {
        set_error("binary16-arithmetic LU: overflow to infinity");
        return NL_ENUMERIC;
    }
    return iflag[0] ? NL_ESINGULAR : NL_OK;
}

extern "C" {

nl_status nl_lu16(int64_t N, void* A16, int64_t ld, int32_t* ipiv, int nb, int gemm, int path, int32_t* info_host,
                  void* stream)
{
    if (N < 1 || N > 32768 || !A16 || !ipiv || ld < N || (ld % 8) || gemm < 0 || gemm > 2 || path < 0 || path > 4) {
        set_error("nl_lu16: bad argument");
        return NL_EINVAL;
    }
    if (path == 3) return lu16_arith_entry((int)N, (__half*)A16, ld, ipiv, info_host, (cudaStream_t)stream);
    if (nb == 0) nb = 128;
    if (!lu16_nb_valid(nb)) {
        set_error("nl_lu16: nb must be a multiple of 16 in [16, 128], or 256, 384 or 512");
        return NL_EINVAL;
    }
    if (gemm == 0) gemm = 2;
    if (gemm == 2 && (nb % 64 || !tc_gemm_supported())) gemm = 1;
    return lu_entry<__half>(N, (__half*)A16, ld, ipiv, nb, gemm, path, info_host, (cudaStream_t)stream, false);
}

nl_status nl_lu64(int64_t N, double* A, int64_t ld, int32_t* ipiv, int nb, int path, int32_t* info_host, void* stream)
{
    if (N < 1 || N > 32768 || !A || !ipiv || ld < N || path < 0 || path > 1) {
        set_error("nl_lu64: bad argument");
        return NL_EINVAL;
    }
    if (nb == 0) nb = 64;
    return lu_entry<double>(N, A, ld, ipiv, nb, 1, path, info_host, (cudaStream_t)stream, true);
}

nl_status nl_lu32(int64_t N, float* A, int64_t ld, int32_t* ipiv, int nb, int32_t* info_host, void* stream)
{
    if (nb == 0) nb = 128;
    if (N < 1 || N > 32768 || !A || !ipiv || ld < N || nb < 16 || nb > 128 || nb % 16) {
        set_error("nl_lu32: bad argument");
        return NL_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int n = (int)N;
    void* wk = nullptr;
    NL_CUDA_OK(cudaMallocAsync(&wk, lu_work_bytes(n, nb, false) + 256, st));
    LuWork w;
    lu_work_carve(wk, n, nb, false, &w);
    int info = 0;
    nl_status s = lu32_factor(n, A, ld, ipiv, nb, w, st, nullptr);
    if (s == NL_OK && cudaMemcpyAsync(&info, w.info, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        s = NL_ECUDA;
    cudaFreeAsync(wk, st);
    NL_CUDA_OK(cudaStreamSynchronize(st));
    if (info_host) *info_host = info;
    if (s == NL_OK && info) return NL_ESINGULAR;
    return s;
}

}  // extern "C"

template <typename S, typename T>
static nl_status lusolve_entry(int64_t N, const S* LU, int64_t ld, const int32_t* ipiv, T* b, void* stream, bool fp64)
{
    if (N < 1 || N > 32768 || !LU || !ipiv || !b || ld < N) {
        set_error("nl_lusolve: bad argument");
        return NL_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int n = (int)N;
    void* wk = nullptr;
    const size_t bytes = trsv_work_bytes(n, fp64);
    NL_CUDA_OK(cudaMallocAsync(&wk, bytes, st));
    NL_CUDA_OK(cudaMemsetAsync(wk, 0, bytes, st));
    TrsvWork w;
    trsv_work_carve(wk, n, fp64, &w);
    nl_status s;
    if constexpr (std::is_same<S, __half>::value) {
        s = trsv_prepare16(n, LU, ld, ipiv, w, st, nullptr);
        if (s == NL_OK) s = trsv_solve16(n, LU, ld, b, b, w, 1, st, nullptr);
    } else if constexpr (std::is_same<S, float>::value) {
        s = trsv_prepare32(n, LU, ld, ipiv, w, st, nullptr);
        if (s == NL_OK) s = trsv_solve32(n, LU, ld, b, b, w, 1, st, nullptr);
    } else {
        s = trsv_prepare64(n, LU, ld, ipiv, w, st, nullptr);
        if (s == NL_OK) s = trsv_solve64(n, LU, ld, b, b, w, 1, st, nullptr);
    }
    unsigned e = 0;
    cudaMemcpyAsync(&e, w.err, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(wk, st);
    NL_CUDA_OK(cudaStreamSynchronize(st));
    if ((s == NL_OK && e) || s == NL_ETIMEOUT) {
        set_error("triangular solve: a bounded wait gave up");
        return NL_ETIMEOUT;
    }
    return s;
}

extern "C" {

nl_status nl_lusolve16(int64_t N, const void* LU16, int64_t ld, const int32_t* ipiv, float* b, void* stream)
{
    return lusolve_entry<__half, float>(N, (const __half*)LU16, ld, ipiv, b, stream, false);
}

nl_status nl_lusolve64(int64_t N, const double* LU, int64_t ld, const int32_t* ipiv, double* b, void* stream)
{
    return lusolve_entry<double, double>(N, LU, ld, ipiv, b, stream, true);
}

nl_status nl_lusolve32(int64_t N, const float* LU, int64_t ld, const int32_t* ipiv, float* b, void* stream)
{
    return lusolve_entry<float, float>(N, LU, ld, ipiv, b, stream, true);  // the 64-row blocked layout
}

nl_status nl_lusolve16h(int64_t N, const void* LU16, int64_t ld, const int32_t* ipiv, void* b16, void* stream)
{
    if (N < 1 || N > 32768 || !LU16 || !ipiv || !b16 || ld < N) {
        set_error("nl_lusolve16h: bad argument");
        return NL_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    __half* b = (__half*)b16;
    NL_TRY(lusolve16h((int)N, (const __half*)LU16, ld, ipiv, nullptr, nullptr, nullptr, nullptr, b, b, nullptr, st));
    NL_CUDA_OK(cudaStreamSynchronize(st));
    return NL_OK;
}

nl_status nl_k_gemv_residual(int64_t N, const float* A, int64_t ld, const float* b, const float* u, float* r,
                             double* rnorm_dev, void* stream)
{
    if (N < 1 || N > 32768 || !A || !u || !r || ld < N) {
        set_error("nl_k_gemv_residual: bad argument");
        return NL_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int n = (int)N;
    const size_t np = gemv_partials(n);
    double* partial = nullptr;
    NL_CUDA_OK(cudaMallocAsync((void**)&partial, sizeof(double) * np + 256, st));
    unsigned* counter = (unsigned*)(partial + np);
    NL_CUDA_OK(cudaMemsetAsync(counter, 0, sizeof(unsigned), st));
    nl_status s = launch_gemv_residual(n, A, ld, b, u, r, partial, counter, rnorm_dev, st);
    cudaFreeAsync(partial, st);
    return s;
}

nl_status nl_k_gemm16_update(int64_t M, int64_t Nc, int64_t K, const void* A, int64_t lda, const void* B, int64_t ldb,
                             void* C, int64_t ldc, int gemm, void* stream)
{
    if (M < 0 || Nc < 0 || K < 1 || !A || !B || !C || gemm < 1 || gemm > 3) {
        set_error("nl_k_gemm16_update: bad argument");
        return NL_EINVAL;
    }
    return gemm16_update((int)M, (int)Nc, (int)K, (const __half*)A, lda, (const __half*)B, ldb, (__half*)C, ldc, gemm,
                         (cudaStream_t)stream);
}

nl_status nl_linsolve16(int64_t N, const float* J32, int64_t ld32, const void* LU16, int64_t ld16, const int32_t* ipiv,
                        const float* b, float* u, double eta, int maxit, int solver, int m, double gtol, int gcycles,
                        int32_t* stats_host, double* relres_host, void* stream)
{
    if (N < 1 || N > 32768 || !J32 || !LU16 || !ipiv || !b || !u || (solver != 0 && solver != 2) || m < 1 || m > 62 ||
        (ld32 % 4) || ld32 < N || ld16 < N) {
        set_error("nl_linsolve16: bad argument");
        return NL_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int n = (int)N;
    const int64_t ldv = round_up(N, 64);
    size_t bytes;
    {
        Carver cv(nullptr);
        for (int q = 0; q < 5; ++q) cv.take<float>(ldv);
        cv.take<float>((size_t)(m + 1) * ldv);
        cv.take<double>(gmres_ws_doubles(m));
        cv.take<double>(gemv_partials(n) + 64);
        cv.take<unsigned>(4);
        cv.take<double>(8);
        cv.take<char>(trsv_work_bytes(n, false));
        bytes = cv.off + 256;
    }
    void* wk = nullptr;
    NL_CUDA_OK(cudaMallocAsync(&wk, bytes, st));
    NL_CUDA_OK(cudaMemsetAsync(wk, 0, bytes, st));
    double* pin = nullptr;
    if (cudaMallocHost((void**)&pin, 64) != cudaSuccess) {
        cudaFreeAsync(wk, st);
        set_error("nl_linsolve16: pinned allocation failed");
        return NL_ENOMEM;
    }
    Carver cv(wk);
    LinBufs B;
    B.r = cv.take<float>(ldv);
    B.d = cv.take<float>(ldv);
    B.t = cv.take<float>(ldv);
    B.w = cv.take<float>(ldv);
    B.ubest = cv.take<float>(ldv);
    B.V = cv.take<float>((size_t)(m + 1) * ldv);
    B.ldv = ldv;
    B.gws = cv.take<double>(gmres_ws_doubles(m));
    B.partial = cv.take<double>(gemv_partials(n) + 64);
    B.counter = cv.take<unsigned>(4);
    B.dscal = cv.take<double>(8);
    TrsvWork tw;
    trsv_work_carve(cv.take<char>(trsv_work_bytes(n, false)), n, false, &tw);
    int launches = 0;
    Host H{pin, st, &launches};
    int epoch = 0;
    LinResult lr;
    nl_status s = trsv_prepare16(n, (const __half*)LU16, ld16, ipiv, tw, st, &launches);
    if (s == NL_OK)
        s = linsolve16(n, J32, ld32, (const __half*)LU16, ld16, tw, epoch, b, u, eta, maxit, solver, m, gtol, gcycles,
                       B, H, &lr);
    unsigned e = 0;
    cudaMemcpyAsync(&e, tw.err, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(wk, st);
    cudaStreamSynchronize(st);
    cudaFreeHost(pin);
    if ((s == NL_OK && e) || s == NL_ETIMEOUT) {
        set_error("triangular solve: a bounded wait gave up");
        return NL_ETIMEOUT;
    }
    if (stats_host) {
        stats_host[0] = lr.iters;
        stats_host[1] = lr.outer;
        stats_host[2] = lr.failed;
        stats_host[3] = lr.converged;
    }
    if (relres_host) *relres_host = lr.relres;
    return s;
}

}  // extern "C"
