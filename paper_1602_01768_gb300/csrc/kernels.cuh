// kernels.cuh -- launchers of the sm_103a kernels (host-callable).
#pragma once
#include "common.cuh"

constexpr int GRAM_CHUNK = 128;  // rows per FP32 Gram partial (summed in FP64)

// api.cu: a handle's device status word and stream
void rb_handle_status(rbfgs_t h, int **status, cudaStream_t *st);

// sketch.cu
template <typename T>
void launch_gauss_sketch(cudaStream_t, int n, int q, uint64_t seed, uint64_t stream, uint64_t k, T *S, int64_t lds);
void launch_coord_trace_draw(cudaStream_t, int n, int q, int nb, const uint64_t *P, uint64_t seed, uint64_t stream,
                             uint64_t k, int *blk);
void launch_floyd_draw(cudaStream_t, int n, int q, uint64_t seed, uint64_t stream, uint64_t k, int *idx);
template <typename T>
void launch_coord_matrix(cudaStream_t, int n, int q, const int *idx, T *S, int64_t lds);
template <typename T>
void launch_block_matrix(cudaStream_t, int n, int q, const int *blk, T *S, int64_t lds);

// gemm_simt.cu: C = alpha op(A) op(B) + beta C (column-major)
template <typename T>
void gemm_simt(cudaStream_t, bool ta, bool tb, int M, int N, int K, T alpha, const T *A, int64_t lda, const T *B,
               int64_t ldb, T beta, T *C, int64_t ldc, const int *status);

// small.cu
template <typename T>
void launch_gram(cudaStream_t, int n, int p, int r, const T *X, int64_t ldx, const T *Y, int64_t ldy, double *part,
                 double *out);
template <typename T>
void launch_core_ada(cudaStream_t, int q, const double *M, const double *N, T *Cinv, T *Dinv, int *status);
void launch_core_ada32(cudaStream_t, int q, const double *M, const double *N, float *Cinv, float *Dinv, int *status);
// q <= 128: X = L^-1 of one FP32 Gram matrix (L L^T = sym(M)), written to
// Xinv (lower, ld q; may be null) and as s1 X^T into xt1 (ld1) and s2 X^T
// into xt2 (ld2) (either may be null).  Returns false for q > 128.
bool launch_core_tr32(cudaStream_t, int q, const float *M, float *Xinv, float *xt1, int ld1, float s1, float *xt2,
                      int ld2, float s2, int *status);
// q <= 128: the same in FP64 (core64.cu): X = L^-1 of sym(M) factored and inverted in
// FP64, written only as the scaled FP32 transposes s1 X^T / s2 X^T; cluster > 1 spreads the
// work over a cluster of that many CTAs (one CTA when no such cluster fits), with the same result.
// Returns the CTAs it launched (0: q > 128 or no launch).
int launch_core_tr64(cudaStream_t, int q, const float *M, float *xt1, int ld1, float s1, float *xt2, int ld2,
                     float s2, int *status, int cluster = 1);
// q <= 64: the RBFGS / AIP core (FP64) from FP32 Gram matrices, packed as the 2q x q B operand
// [B1; -Lam] (Tf given: RBFGS) or [Lam; -Lam] (Tf null: AIP), ld 2q; scratch: 3 q^2 doubles.
void launch_core_pack(cudaStream_t, int q, const float *Mf, const float *Tf, float *Bw, double *scratch,
                      int *status);
// out[off + c + i rp] = X[i + c ldx] for i < n, c < q: a column-major panel into rows of pitch rp.
void launch_rows_from_cols(cudaStream_t, int n, int q, const float *X, int64_t ldx, float *out, int rp, int off);
template <typename T>
void launch_core_rbfgs(cudaStream_t, int q, const double *M, const double *Tm, T *Lam, T *B1, int *status);
template <typename T>
void launch_set_identity(cudaStream_t, int n, T *X, int64_t ld, T diag);
template <typename Ti, typename To>
void launch_copy2d(cudaStream_t, int rows, int cols, const Ti *X, int64_t ldx, To *Y, int64_t ldy, double alpha);
template <typename T>
void launch_diag(cudaStream_t, int n, const T *A, int64_t lda, double *d);

// aux.cu
template <typename T>
void launch_resid_sumsq(cudaStream_t, int n, int m, const T *Z, int64_t ldz, const int *J, double *part,
                        double *out);
template <typename T>
void launch_gather_cols(cudaStream_t, int n, int m, const T *A, int64_t lda, const int *J, T *Y, int64_t ldy);
template <typename T>
void launch_coord_gather(cudaStream_t, int n, int q, const T *A, int64_t lda, const int *blk, T *G, int64_t ldg,
                         double *Mpad, const int *status);
template <typename T>
void launch_coord_add_b1(cudaStream_t, int q, const int *blk, const T *B1, T *W, int64_t ldw, const int *status);
// AIP with a coordinate block: V[:, C] += Lambda, then X[C, :] += V (first size rows).
template <typename T>
void launch_aip_coord(cudaStream_t, int n, int q, const int *blk, const T *Lam, T *V, int64_t ldv, T *X, int64_t ldx,
                      const int *status);
template <typename T>
void launch_coord_update(cudaStream_t, int n, int q, const int *blk, const T *W, int64_t ldw, T *X, int64_t ldx,
                         const int *status);
template <typename T>
void launch_mr_dots(cudaStream_t, int n, const T *P, int64_t ldp, const T *Q, int64_t ldq, double *part,
                    double *out);
template <typename T>
void launch_i_minus(cudaStream_t, int n, T *P, int64_t ld);
template <typename T>
void launch_axpy_dev(cudaStream_t, int n, const double *dots, const T *D, int64_t ldd, T *X, int64_t ldx);
template <typename T>
void launch_power_iteration(cudaStream_t, int n, const T *A, int64_t lda, int iters, double *v, double *w,
                            double *sigma);
