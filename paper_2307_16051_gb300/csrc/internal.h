// internal.h — launchers shared between the translation units of the library.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <vector>

#include "../../include/newton3p.h"

namespace nl {

// problem.cu
nl_status launch_htab(int N, double* htab, cudaStream_t st);
nl_status launch_residual(int N, double c, const double* x, const void* u, int u_is_double, double scale,
                          const double* htab, double* xout, double* F, double* rr, double* partial,
                          unsigned* counter, double* fnorm, cudaStream_t st);
int residual_partials(int N);

// fft.cu: the residual of eq. (3.2) through a length-L FFT convolution (L the
// power of two >= max(4, 2N), split L = L1 L2 for the two passes).
struct FftPlan {
    int N = 0, L = 0, L1 = 0, L2 = 0;
    double2* tw = nullptr;   // L twiddles exp(-2 pi i k / L)
    double2* Hh = nullptr;   // transform of h[k] = 1/(k+1), k < 2N-1, zero-padded
    double2* Y = nullptr;    // work: L
    double2* V = nullptr;    // work: L
    double* part = nullptr;  // L1 per-block partial sums of F_i^2
    unsigned* cnt = nullptr; // finishing counter (zero between calls)
};
size_t fft_work_bytes(int N);
void fft_work_carve(void* base, int N, FftPlan* p);
nl_status fft_prepare(const FftPlan& p, cudaStream_t st);  // twiddles and Hh (once per plan)
// As launch_residual (same outputs, norm deterministic), O(N log N).
nl_status launch_residual_fft(const FftPlan& p, double c, const double* x, const void* u, int u_is_double,
                              double scale, double* xout, double* F, double* rr, double* fnorm, cudaStream_t st);
// rs != NULL: J16 scaled into the binary16 range row by row (power-of-two
// factors written to rs[0..N)); see k_jacobian.
nl_status launch_jacobian(int N, double c, const double* rr, const double* htab, float* J32, int64_t ld32,
                          __half* J16, int64_t ld16, cudaStream_t st, float* rs = nullptr);
nl_status launch_jacobian64(int N, double c, const double* rr, const double* htab, double* J, int64_t ld,
                            cudaStream_t st);

// lu.cu: blocked LU with partial pivoting.
struct LuWork {
    void* pnl = nullptr;      // outer-panel working copy: N x NB (float for fp16 LU, double for fp64 LU)
    __half* ut = nullptr;     // U12^T for the tensor-core trailing update: N x NB binary16
    int* info = nullptr;      // device int: first zero pivot (1-based), 0 if none; the 256-byte info block
                              // also holds the flag (+1), an error word (+2), the binary16-arithmetic LU's
                              // barrier (+4, +5) and the streaming panel's two role counters (+8, +9)
    int* flag = nullptr;      // device int (info + 1): set when the no-interchange fast path failed
    void* stage = nullptr;    // diagonal-block factors staged for the off-diagonal solves (<= 256 KB)
    unsigned long long* pub = nullptr;  // 128 x 128 {epoch, value} words: columns published by k_panel16
    int stream = 0;           // binary16 fast path: 0 = one streaming launch per panel when it fits (128 rows per
                              // CTA when possible), 256 = the same with 256 rows per CTA, -1 = two launches
    float* p32 = nullptr;     // two-level LU (outer block > 128): single-precision shadow of the matrix, N x ldp32,
                              // of which the current outer block's row and column strips are used
    int64_t ldp32 = 0;
    // Look-ahead (one-level binary16 fast path with the tensor-core update): after panel p the
    // next panel's row and column strips are updated on the caller's stream (or by the next
    // panel's own CTAs), the rest of the trailing matrix on side, joined before the next
    // panel's strips are updated again.  ut2: the second
    // U12^T buffer (panels alternate, so panel p + 1 never writes what the update of panel p
    // reads).  Owned by whoever set them; no look-ahead while side is null.
    __half* ut2 = nullptr;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join[2] = {nullptr, nullptr};  // ev_join[q % 2]: the rest of update q
};
// The look-ahead's side stream and events for w (created at st's priority, or
// re-created when the priority differs); lu_side_release destroys them.
nl_status lu_side_prepare(LuWork* w, cudaStream_t st);
void lu_side_release(LuWork* w);
size_t lu_work_bytes(int N, int nb, bool fp64);
void lu_work_carve(void* base, int N, int nb, bool fp64, LuWork* w);
// gemm: 1 = SIMT, 2 = tcgen05.  Asynchronous; *info is written on the device.
// fast: factor without interchanges, checking on every pre-division value that
// partial pivoting would keep the diagonal; the result equals partial pivoting
// when *flag stays 0, otherwise A is left partly factored and the caller
// restores A and calls again with fast = false.
// nb: a multiple of 16 up to 128 (one level), or 256, 384, 512 (two levels,
// fast path; lu16_nb_valid).
bool lu16_nb_valid(int nb);
nl_status lu16_factor(int N, __half* A, int64_t ld, int* ipiv, int nb, int gemm, bool fast, const LuWork& w,
                      cudaStream_t st, int* launches);
nl_status lu64_factor(int N, double* A, int64_t ld, int* ipiv, int nb, bool fast, const LuWork& w, cudaStream_t st,
                      int* launches);
// Binary32 storage and arithmetic (F32 Newton), always with interchanges;
// w carved for the single-precision panel (fp64 = false).
nl_status lu32_factor(int N, float* A, int64_t ld, int* ipiv, int nb, const LuWork& w, cudaStream_t st, int* launches);
// Every operation rounded to binary16 (the F16 column's arithmetic), partial
// pivoting, one cooperative launch.  Asynchronous: w.info[0] = first zero
// pivot (1-based) or 0, w.info[1] != 0 after a binary16 overflow; a barrier
// that gave up sets the tensor-core error word (or w.info[2]).
nl_status lu16_factor_arith(int N, __half* A, int64_t ld, int* ipiv, const LuWork& w, cudaStream_t st);
nl_status gemm16_update(int M, int Nc, int K, const __half* A, int64_t lda, const __half* B, int64_t ldb,
                        __half* C, int64_t ldc, int gemm, cudaStream_t st);

// Grouped LU (many independent matrices, one launch per kernel class per
// outer step).  The instance table lives in device memory.
struct GInst {
    void* A;        // binary16 or double matrix, row-major, leading dimension ld
    int64_t ld;
    int N;
    int pad;
    int* ipiv;      // N
    int* flag;      // bit 0: the no-interchange fast path failed; bit 1: skip this matrix
    void* stage;    // diagonal-block staging (lu_stage_bytes)
    __half* ut;     // U12^T buffer for the tensor-core update: round_up(N, 128) x nb binary16
};
struct GTask {      // diag: {inst}; offdiag: {inst, block, row blocks}; gemm: {inst, m0, n0}
    int inst, a, b, pad;
};
struct alignas(64) TmapBytes {  // an opaque CUtensorMap
    unsigned char b[128];
};
// Per-step task lists of a grouped factorisation (device arrays, owned).
struct PTask;
struct GroupPlan {
    int count = 0, nb = 128, gemm = 1, steps = 0;
    bool fp64 = false;
    int kind = 0;              // 0: three launches per outer step; 1: one persistent launch (task queue)
    int tm = 64, tn = 64;      // kind 1: update tile (SIMT: tm x 64, tm 64 or 128; tcgen05: 128 x 128)
    std::vector<int> off, n;   // per step and class (3 * steps): offset into tasks and count
    GTask* tasks = nullptr;    // device
    TmapBytes* maps = nullptr; // device: 2 per instance (A and U12^T views), tensor-core update only
    PTask* ptasks = nullptr;   // kind 1: the queue (device)
    int nptasks = 0, grid = 0;
    int* ctl = nullptr;        // kind 1: next-task counter, progress words, task counters (zeroed per launch)
    size_t bytes = 0;
};
size_t lu_stage_bytes();
// Builds the plan for the instances (host copy of the device table, which must
// already hold final pointers).  Allocates the device task and map arrays.
// kind 1 (one persistent launch over a device task queue) needs the binary16
// factorisation and nb <= 64: gemm 1 SIMT update tiles of tm x 64, gemm 2
// tcgen05 tiles of 128 x 128 (nb = 64).
nl_status lu_grouped_plan(int count, const GInst* host_inst, int nb, int gemm, bool fp64, GroupPlan* plan,
                          int kind = 0, int tm = 64);
void lu_grouped_free(GroupPlan* plan);
// One-time kernel attribute set-up (call before any stream capture).
nl_status lu_grouped_setup();
// Launches the whole factorisation (kind 0: 3 launches per outer step; kind 1: a
// memset and one launch); stream-capturable.
nl_status lu_grouped_factor(const GroupPlan& plan, const GInst* dev_inst, cudaStream_t st, int* launches);

// Batched Newton (batch.cu): one instance of the H-equation per entry.
enum : int {
    BS_ACTIVE = 0,     // Newton continues
    BS_CONVERGED = 1,  // ||F|| <= tau
    BS_PARKED_LU = 2,  // the factorisation needs row interchanges: finished on the single-instance path
    BS_PARKED_IR = 3,  // IR stalled: finished on the single-instance path with GMRES-IR
    BS_NOTCONV = 4,    // Newton cap reached
    BS_NUMERIC = 5     // non-finite residual
};
struct BInst {
    int N, ld;         // ld: row stride of J32 and J (multiple of 64)
    double c;
    double* x[2];      // iterate buffers; BState::par selects the current one
    double *F, *rr;
    float* J32;
    void* J;           // binary16 (three-precision) or double (FP64 mode) Jacobian, factored in place
    int* ipiv;
    int* flag;         // the grouped LU's flag word
    float *b, *u, *r;  // single-precision IR vectors (ld entries)
    double *b64, *u64; // double step (FP64 mode)
    double* part;      // per-block partial sums of the norms
    unsigned* cnt;     // [0] residual blocks done, [1] residual-GEMV blocks done
    const double* x0;
    double* xout;      // slice of the packed output
};
struct BState {
    int status, it, par, lin_active;
    int outer, lin_iters, failed, pad;
    double fn0, fn, tau, nb, nr, prev, nr_new, pad2;
};
struct BTask {         // a block of rows of one instance
    int inst, i0;
};
int residual_block_rows();  // rows per block of the grouped residual
int gemv_block_rows();      // rows per block of the grouped residual GEMV
// mode 0: F at x[0] (every instance); 1: x[par^1] = x[par] + fn u (single u), then F; 2: the same with u64.
// Modes 1 and 2 skip instances that are not BS_ACTIVE.  The last block of an instance writes st.fn.
nl_status launch_residual_g(const BInst* inst, BState* st, const BTask* tasks, int ntasks, int mode,
                            const double* htab, cudaStream_t st_);
// J32/J16 (fp64 = 0) or J64 (fp64 = 1) of the BS_ACTIVE instances; rows = total rows, row_off[count + 1].
nl_status launch_jacobian_g(const BInst* inst, const BState* st, const int* row_off, int count, int rows,
                            const double* htab, const float* htab32, int fp64, cudaStream_t st_);
// r = b - J32 u of instances with lin_active; the last block of an instance writes st.nr_new.
nl_status launch_gemv_residual_g(const BInst* inst, BState* st, const BTask* tasks, int ntasks, cudaStream_t st_);

// gemm_tc.cu: C = fl16(C - A * Bt^T), A M x K (lda), Bt Nc x K (ldbt), tcgen05 + TMA.
// cross: only the first 128-column tile column and the first 128-row tile row of C.
// max_ctas > 0 caps the grid of a small shallow update (K < 256, at most 8 tiles per SM).
bool tc_gemm_supported();
// C <- C - A B on the tensor cores for binary32 C and binary32 operands holding
// binary16 values (the two-level LU's inner updates), K <= 128, any M, Nc.
nl_status tc_update_f32(int M, int Nc, int K, const float* A, int64_t lda, const float* B, int64_t ldb, float* C,
                        int64_t ldc, cudaStream_t st, const int* flag);
nl_status tc_gemm16_update(int M, int Nc, int K, const __half* A, int64_t lda, const __half* Bt, int64_t ldbt,
                           __half* C, int64_t ldc, cudaStream_t st, const int* flag, bool per_tile = false,
                           bool cross = false, int max_ctas = 0);

// trsv.cu: triangular solves with the factors.
constexpr int kTrsvT = 64;  // diagonal block size
struct TrsvWork {
    int* perm = nullptr;      // N: position -> original index
    void* dinv = nullptr;     // 2 * nblk * T * T elements (float or double): inverses of L_bb and U_bb
    int* flags = nullptr;     // 2 * nblk ints, epoch-tagged readiness flags
    void* y = nullptr;        // N elements: forward-solve result
    unsigned* err = nullptr;  // device error word
    int* scan = nullptr;      // scratch for the permutation build
    int cluster = 0;          // half-precision solve: 0 = largest cluster available, -1 = mailbox kernel, else cap
    const float* rs = nullptr;  // half-precision solve: row factors of a factorisation of R J (the right side
                                // is multiplied by R first), or null
    int wait_limit = 0;       // half-precision solve's waits: 0 = default bound (about a second), < 0 = give up at
                              // once (test of the timeout path), > 0 = polls (cluster) / cycles (mailbox)
};
size_t trsv_work_bytes(int N, bool fp64);
void trsv_work_carve(void* base, int N, bool fp64, TrsvWork* w);
nl_status trsv_prepare16(int N, const __half* LU, int64_t ld, const int* ipiv, const TrsvWork& w, cudaStream_t st,
                         int* launches);
nl_status trsv_prepare64(int N, const double* LU, int64_t ld, const int* ipiv, const TrsvWork& w, cudaStream_t st,
                         int* launches);
// z = U^{-1} L^{-1} P v (v, z may alias).  epoch: strictly increasing per call on the same workspace.
nl_status trsv_solve16(int N, const __half* LU, int64_t ld, const float* v, float* z, const TrsvWork& w, int epoch,
                       cudaStream_t st, int* launches);
nl_status trsv_solve64(int N, const double* LU, int64_t ld, const double* v, double* z, const TrsvWork& w, int epoch,
                       cudaStream_t st, int* launches);
// Single-precision factors (F32 Newton): the blocked solve of the double path
// in binary32, so w is carved with the double layout (fp64 = true).
nl_status trsv_prepare32(int N, const float* LU, int64_t ld, const int* ipiv, const TrsvWork& w, cudaStream_t st,
                         int* launches);
nl_status trsv_solve32(int N, const float* LU, int64_t ld, const float* v, float* z, const TrsvWork& w, int epoch,
                       cudaStream_t st, int* launches);
// B = A (N x N binary16 promoted to binary32, exact).
nl_status launch_promote16(int N, const __half* A, int64_t lda, float* B, int64_t ldb, cudaStream_t st);
// Both triangular solves in binary16 arithmetic, z = U^{-1} L^{-1} P v, on
//   v = fl16(-F / *nrm)  when F is given (the F16 Newton step, eq. (2.17)),
//   v = fl16(r / rn)     when r is given, rn = fl32(*nrm) (eq. (2.19)),
//   v = vin              otherwise (binary16).
// P from perm (position -> original index, as trsv_prepare16 builds it) when
// given, else from the interchanges ipiv.  The result goes to zout (binary16)
// and / or u (binary32: z, or rn z when r is given); either may be null.
// One CTA; N <= 32768.
nl_status lusolve16h(int N, const __half* LU, int64_t ld, const int* ipiv, const int* perm, const double* F,
                     const float* r, const double* nrm, const __half* vin, __half* zout, float* u, cudaStream_t st);

// krylov.cu
nl_status launch_gemv_residual(int N, const float* A, int64_t ld, const float* b, const float* u, float* r,
                               double* partial, unsigned* counter, double* rnorm, cudaStream_t st);
int gemv_partials(int N);
nl_status launch_scale_rhs32(int N, const double* F, const double* fnorm, float* b, cudaStream_t st);
nl_status launch_scale_rhs64(int N, const double* F, const double* fnorm, double* b, cudaStream_t st);
nl_status launch_axpy32(int N, float a, const float* x, float* y, cudaStream_t st);
nl_status launch_norm32(int N, const float* v, double* partial, unsigned* counter, double* out, cudaStream_t st);
// GMRES pieces: V is (m+1) x N; ws holds the Hessenberg/Givens state in double.
// ws scalars (doubles at ws + gmres_scal_offset(m)): {beta, residual estimate, breakdown}.
int gmres_ws_doubles(int m);
int gmres_scal_offset(int m);
nl_status launch_gmres_start(int N, const float* z, float* V, double* ws, int m, cudaStream_t st);
nl_status launch_arnoldi(int N, int64_t ldv, float* w, float* V, int j, double* ws, int m, cudaStream_t st);
nl_status launch_gmres_update(int N, int64_t ldv, const float* V, double* ws, int m, int jcols, float* d,
                              cudaStream_t st);
unsigned* tc_error_word();
// Tensor maps of one grouped instance: the whole N x N binary16 matrix (ld)
// and its U12^T buffer (round_up(N, 128) x nb), 64 x 128 boxes.
bool tc_encode_instance_maps(const __half* A, int N, int64_t ld, const __half* ut, int nb, TmapBytes* out2);
// Grouped trailing update of one outer step [K, K + w): tasks {inst, m0, n0}.
nl_status tc_gemm16_grouped(const GInst* inst, const TmapBytes* maps, const GTask* tasks, int ntasks, int K, int w,
                            cudaStream_t st);

}  // namespace nl
