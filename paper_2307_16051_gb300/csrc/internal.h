// internal.h — launchers shared between the translation units of the library.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "../../include/newton3p.h"

namespace nl {

// problem.cu
nl_status launch_htab(int N, double* htab, cudaStream_t st);
nl_status launch_residual(int N, double c, const double* x, const void* u, int u_is_double, double scale,
                          const double* htab, double* xout, double* F, double* rr, double* partial,
                          unsigned* counter, double* fnorm, cudaStream_t st);
int residual_partials(int N);
nl_status launch_jacobian(int N, double c, const double* rr, const double* htab, float* J32, int64_t ld32,
                          __half* J16, int64_t ld16, cudaStream_t st);
nl_status launch_jacobian64(int N, double c, const double* rr, const double* htab, double* J, int64_t ld,
                            cudaStream_t st);

// lu.cu: blocked LU with partial pivoting.
struct LuWork {
    void* pnl = nullptr;      // outer-panel working copy: N x NB (float for fp16 LU, double for fp64 LU)
    __half* ut = nullptr;     // U12^T for the tensor-core trailing update: N x NB binary16
    int* info = nullptr;      // device int: first zero pivot (1-based), 0 if none
    int* flag = nullptr;      // device int (info + 1): set when the no-interchange fast path failed
    void* stage = nullptr;    // diagonal-block factors staged for the off-diagonal solves (<= 256 KB)
};
size_t lu_work_bytes(int N, int nb, bool fp64);
void lu_work_carve(void* base, int N, int nb, bool fp64, LuWork* w);
// gemm: 1 = SIMT, 2 = tcgen05.  Asynchronous; *info is written on the device.
// fast: factor without interchanges, checking on every pre-division value that
// partial pivoting would keep the diagonal; the result equals partial pivoting
// when *flag stays 0, otherwise A is left partly factored and the caller
// restores A and calls again with fast = false.
nl_status lu16_factor(int N, __half* A, int64_t ld, int* ipiv, int nb, int gemm, bool fast, const LuWork& w,
                      cudaStream_t st, int* launches);
nl_status lu64_factor(int N, double* A, int64_t ld, int* ipiv, int nb, bool fast, const LuWork& w, cudaStream_t st,
                      int* launches);
nl_status gemm16_update(int M, int Nc, int K, const __half* A, int64_t lda, const __half* B, int64_t ldb,
                        __half* C, int64_t ldc, int gemm, cudaStream_t st);

// gemm_tc.cu: C = fl16(C - A * Bt^T), A M x K (lda), Bt Nc x K (ldbt), tcgen05 + TMA.
bool tc_gemm_supported();
nl_status tc_gemm16_update(int M, int Nc, int K, const __half* A, int64_t lda, const __half* Bt, int64_t ldbt,
                           __half* C, int64_t ldc, cudaStream_t st, const int* flag);

// trsv.cu: triangular solves with the factors.
constexpr int kTrsvT = 64;  // diagonal block size
struct TrsvWork {
    int* perm = nullptr;      // N: position -> original index
    void* dinv = nullptr;     // 2 * nblk * T * T elements (float or double): inverses of L_bb and U_bb
    int* flags = nullptr;     // 2 * nblk ints, epoch-tagged readiness flags
    void* y = nullptr;        // N elements: forward-solve result
    unsigned* err = nullptr;  // device error word
    int* scan = nullptr;      // scratch for the permutation build
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

}  // namespace nl
