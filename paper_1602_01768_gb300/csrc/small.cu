// small.cu -- the q x q core of each step and the small helpers around it.
//
//  * Gram products X^T Y of two n x q panels (S^T A S, S~^T S~, G^T X G):
//    FP32 (or FP64) products summed over row chunks of GRAM_CHUNK rows, the
//    chunk partials summed in FP64 in a fixed order (deterministic).
//  * FP64 q x q core, one CTA per matrix with the matrix in shared memory:
//    lower Cholesky (a pivot <= 0 or non-finite sets ST_NOTSPD) and the
//    inverse of the triangular factor.
#include "kernels.cuh"

// ---------------------------------------------------------------------------
// Gram partials: part[c][i + j p] = sum over rows of chunk c of X[row, i] Y[row, j]
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_gram_partial(int n, int p, int r, const T *__restrict__ X, int64_t ldx,
                                                      const T *__restrict__ Y, int64_t ldy, double *part)
{
    __shared__ T xs[32][33];
    __shared__ T ys[32][33];
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    const int row0 = blockIdx.z * GRAM_CHUNK;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (int rb = row0; rb < row0 + GRAM_CHUNK && rb < n; rb += 32) {
        for (int e = threadIdx.x; e < 32 * 32; e += 256) {
            const int rr = e & 31, cc = e >> 5;
            const int row = rb + rr;
            xs[cc][rr] = (row < n && i0 + cc < p) ? X[row + (int64_t)(i0 + cc) * ldx] : T(0);
            ys[cc][rr] = (row < n && j0 + cc < r) ? Y[row + (int64_t)(j0 + cc) * ldy] : T(0);
        }
        __syncthreads();
#pragma unroll 8
        for (int rr = 0; rr < 32; ++rr) {
            const T xv = xs[tx][rr];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = fma(xv, ys[ty + 8 * u][rr], acc[u]);
        }
        __syncthreads();
    }
    double *out = part + (size_t)blockIdx.z * p * r;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int i = i0 + tx, j = j0 + ty + 8 * u;
        if (i < p && j < r) out[i + (size_t)j * p] = (double)acc[u];
    }
}

// out[e] = sum_c part[c][e] in a fixed order: thread group g of 8 sums the
// chunks c = g, g + 8, ... (independent loads issued together), then the 8
// group sums are added in order g = 0..7.  Deterministic and not latency bound.
__global__ void __launch_bounds__(256) k_gram_reduce(int nchunks, int pr, const double *part, double *out)
{
    __shared__ double red[8][33];
    const int o = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int e = blockIdx.x * 32 + o;
    double s = 0.0;
    if (e < pr) {
        int c = g;
        for (; c + 24 < nchunks; c += 32) {  // four independent loads in flight
            const double a0 = part[(size_t)c * pr + e], a1 = part[(size_t)(c + 8) * pr + e];
            const double a2 = part[(size_t)(c + 16) * pr + e], a3 = part[(size_t)(c + 24) * pr + e];
            s += a0;
            s += a1;
            s += a2;
            s += a3;
        }
        for (; c < nchunks; c += 8) s += part[(size_t)c * pr + e];
    }
    red[g][o] = s;
    __syncthreads();
    if (g == 0 && e < pr) {
        double t = 0.0;
        for (int k = 0; k < 8; ++k) t += red[k][o];
        out[e] = t;
    }
}

// One CTA per GRAM_CHUNK rows computing all p x r outputs (p, r <= 128):
// rows are staged 32 at a time in shared memory; thread (tx, ty) of a 16 x 16
// grid owns outputs (ty + 16 a, tx + 16 b).  FP32 products summed over the
// chunk, written as one FP64 partial per chunk.
template <typename T>
__global__ void __launch_bounds__(256) k_gram_chunk(int n, int p, int r, const T *__restrict__ X, int64_t ldx,
                                                    const T *__restrict__ Y, int64_t ldy, double *part)
{
    __shared__ T xs[32][128 + 4];
    __shared__ T ys[32][128 + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int row0 = blockIdx.x * GRAM_CHUNK;
    T acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = T(0);
    for (int rb = row0; rb < row0 + GRAM_CHUNK && rb < n; rb += 32) {
        for (int e = threadIdx.x; e < 32 * 128; e += 256) {
            const int rr = e & 31, cc = e >> 5;
            const int row = rb + rr;
            xs[rr][cc] = (row < n && cc < p) ? X[row + (int64_t)cc * ldx] : T(0);
            ys[rr][cc] = (row < n && cc < r) ? Y[row + (int64_t)cc * ldy] : T(0);
        }
        __syncthreads();
#pragma unroll 4
        for (int rr = 0; rr < 32; ++rr) {
            T xv[8], yv[8];
#pragma unroll
            for (int a = 0; a < 8; ++a) xv[a] = xs[rr][ty + 16 * a];
#pragma unroll
            for (int b = 0; b < 8; ++b) yv[b] = ys[rr][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[a][b] = fma(xv[a], yv[b], acc[a][b]);
        }
        __syncthreads();
    }
    double *out = part + (size_t)blockIdx.x * p * r;
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int i = ty + 16 * a, j = tx + 16 * b;
            if (i < p && j < r) out[i + (size_t)j * p] = (double)acc[a][b];
        }
}

template <typename T>
void launch_gram(cudaStream_t st, int n, int p, int r, const T *X, int64_t ldx, const T *Y, int64_t ldy,
                 double *part, double *out)
{
    const int nch = ceil_div(n, GRAM_CHUNK);
    if constexpr (sizeof(T) == 4) {
        if (p <= 128 && r <= 128) {
            rb_count_launch();
            k_gram_chunk<T><<<nch, 256, 0, st>>>(n, p, r, X, ldx, Y, ldy, part);
            rb_count_launch();
            k_gram_reduce<<<ceil_div(p * r, 32), 256, 0, st>>>(nch, p * r, part, out);
            return;
        }
    }
    dim3 grid(ceil_div(p, 32), ceil_div(r, 32), nch);
    rb_count_launch();
    k_gram_partial<T><<<grid, 256, 0, st>>>(n, p, r, X, ldx, Y, ldy, part);
    rb_count_launch();
    k_gram_reduce<<<ceil_div(p * r, 32), 256, 0, st>>>(nch, p * r, part, out);
}
template void launch_gram<float>(cudaStream_t, int, int, int, const float *, int64_t, const float *, int64_t,
                                 double *, double *);
template void launch_gram<double>(cudaStream_t, int, int, int, const double *, int64_t, const double *, int64_t,
                                  double *, double *);

// ---------------------------------------------------------------------------
// FP64 core in shared memory.
// ---------------------------------------------------------------------------

// Right-looking lower Cholesky of a (q x q, column-major, in smem).  Returns
// false on a pivot <= 0 or non-finite (all threads agree).
__device__ bool smem_cholesky(double *a, int q)
{
    __shared__ int fail;
    if (threadIdx.x == 0) fail = 0;
    __syncthreads();
    for (int j = 0; j < q; ++j) {
        if (threadIdx.x == 0) {
            const double d = a[j + j * q];
            if (!(d > 0.0) || !isfinite(d))
                fail = 1;
            else
                a[j + j * q] = sqrt(d);
        }
        __syncthreads();
        if (fail) return false;
        const double piv = a[j + j * q];
        for (int i = j + 1 + threadIdx.x; i < q; i += blockDim.x) a[i + j * q] /= piv;
        __syncthreads();
        // trailing update of the lower triangle: a[i][c] -= a[i][j] a[c][j], j < c <= i
        const int m = q - j - 1;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const int c = j + 1 + e / m, i = j + 1 + e % m;
            if (i >= c) a[i + c * q] -= a[i + j * q] * a[c + j * q];
        }
        __syncthreads();
    }
    // zero the strict upper triangle
    for (int e = threadIdx.x; e < q * q; e += blockDim.x) {
        const int i = e % q, c = e / q;
        if (i < c) a[e] = 0.0;
    }
    __syncthreads();
    return true;
}

// In-place inverse of a lower-triangular matrix.  Column c of X = L^-1:
// X_cc = 1/L_cc, X_ic = -(sum_{k=c}^{i-1} L_ik X_kc) / L_ii.  Columns are
// independent (one thread each); X_ic is first written to the unused upper
// slot (c, i) so the lower entries L_ik other threads read stay intact, then
// transposed down.
__device__ void smem_tri_inverse(double *a, int q)
{
    for (int c = threadIdx.x; c < q; c += blockDim.x) a[c + c * q] = 1.0 / a[c + c * q];
    __syncthreads();
    for (int c = threadIdx.x; c < q; c += blockDim.x) {
        for (int i = c + 1; i < q; ++i) {
            double s = a[i + c * q] * a[c + c * q];
            for (int k = c + 1; k < i; ++k) s += a[i + k * q] * a[c + k * q];
            a[c + i * q] = -s * a[i + i * q];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < q * q; e += blockDim.x) {
        const int i = e % q, c = e / q;
        if (i > c) a[e] = a[c + i * q];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < q * q; e += blockDim.x) {
        const int i = e % q, c = e / q;
        if (i < c) a[e] = 0.0;
    }
    __syncthreads();
}

// AdaRBFGS core: blockIdx.x = 0 factors M = S^T A S -> C and writes C^-1;
// blockIdx.x = 1 factors N = S~^T S~ -> D and writes D^-1 (both lower, T).
template <typename T>
__global__ void k_core_ada(int q, const double *M, const double *N, T *Cinv, T *Dinv, int *status)
{
    extern __shared__ double sm[];
    if (status_bad(status)) return;
    const double *src = blockIdx.x == 0 ? M : N;
    T *dst = blockIdx.x == 0 ? Cinv : Dinv;
    for (int e = threadIdx.x; e < q * q; e += blockDim.x) {
        const int i = e % q, c = e / q;
        // symmetrise the computed Gram from its two triangles
        sm[e] = 0.5 * (src[i + c * q] + src[c + i * q]);
    }
    __syncthreads();
    if (!smem_cholesky(sm, q)) {
        if (threadIdx.x == 0) atomicOr(status, ST_NOTSPD);
        return;
    }
    smem_tri_inverse(sm, q);
    for (int e = threadIdx.x; e < q * q; e += blockDim.x) {
        const int i = e % q, c = e / q;
        dst[e] = (T)(i >= c ? sm[e] : 0.0);
    }
}

template <typename T>
void launch_core_ada(cudaStream_t st, int q, const double *M, const double *N, T *Cinv, T *Dinv, int *status)
{
    const size_t smem = sizeof(double) * q * q;
    static bool attr_set = false;  // idempotent: the attribute is per function
    if (!attr_set) {
        cudaFuncSetAttribute(k_core_ada<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        attr_set = true;
    }
    rb_count_launch();
    k_core_ada<T><<<2, 512, smem, st>>>(q, M, N, Cinv, Dinv, status);
}
template void launch_core_ada<float>(cudaStream_t, int, const double *, const double *, float *, float *, int *);
template void launch_core_ada<double>(cudaStream_t, int, const double *, const double *, double *, double *,
                                      int *);

// RBFGS core: C C^T = M, Lam = C^-T C^-1, B1 = (Lam + Lam T Lam)/2.  One CTA.
template <typename T>
__global__ void k_core_rbfgs(int q, const double *M, const double *Tm, T *Lam_out, T *B1_out, int *status)
{
    extern __shared__ double sm[];
    double *a = sm;              // C, then C^-1
    double *lam = sm + q * q;    // Lam
    double *tl = sm + 2 * q * q; // T Lam
    if (status_bad(status)) return;
    for (int e = threadIdx.x; e < q * q; e += blockDim.x) {
        const int i = e % q, c = e / q;
        a[e] = 0.5 * (M[i + c * q] + M[c + i * q]);
    }
    __syncthreads();
    if (!smem_cholesky(a, q)) {
        if (threadIdx.x == 0) atomicOr(status, ST_NOTSPD);
        return;
    }
    smem_tri_inverse(a, q);
    // Lam = C^-T C^-1: Lam_ij = sum_k Cinv_ki Cinv_kj (k >= max(i, j))
    for (int e = threadIdx.x; e < q * q; e += blockDim.x) {
        const int i = e % q, j = e / q;
        double s = 0.0;
        for (int k = max(i, j); k < q; ++k) s += a[k + i * q] * a[k + j * q];
        lam[e] = s;
    }
    __syncthreads();
    // T Lam (T symmetrised)
    for (int e = threadIdx.x; e < q * q; e += blockDim.x) {
        const int i = e % q, j = e / q;
        double s = 0.0;
        for (int k = 0; k < q; ++k) s += 0.5 * (Tm[i + k * q] + Tm[k + i * q]) * lam[k + j * q];
        tl[e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < q * q; e += blockDim.x) {
        const int i = e % q, j = e / q;
        double s = 0.0;
        for (int k = 0; k < q; ++k) s += lam[i + k * q] * tl[k + j * q];
        const double b1 = 0.5 * (lam[e] + s);
        if (!isfinite(b1)) atomicOr(status, ST_NONFINITE);
        B1_out[e] = (T)b1;
        Lam_out[e] = (T)lam[e];
    }
}

template <typename T>
void launch_core_rbfgs(cudaStream_t st, int q, const double *M, const double *Tm, T *Lam, T *B1, int *status)
{
    const size_t smem = sizeof(double) * 3 * q * q;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_core_rbfgs<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        attr_set = true;
    }
    rb_count_launch();
    k_core_rbfgs<T><<<1, 512, smem, st>>>(q, M, Tm, Lam, B1, status);
}
template void launch_core_rbfgs<float>(cudaStream_t, int, const double *, const double *, float *, float *, int *);
template void launch_core_rbfgs<double>(cudaStream_t, int, const double *, const double *, double *, double *,
                                        int *);

// Tensor-core forms of RBFGS and AIP: the same FP64 core from FP32 Gram matrices
// (M = S^T A S and, for RBFGS, T = G^T X G), written straight into the
// 2q x q B operand (ld 2q) of the product that forms the update's panel:
//   RBFGS (Tf != null): [B1; -Lam], B1 = (Lam + Lam T Lam) / 2, for W = [S | Y] [B1; -Lam];
//   AIP   (Tf == null): [Lam; -Lam], for V^T = [S | W^T] [Lam; -Lam].
// GB300 runs FP64 at a small fraction of its FP32 rate, so only the factorisation
// stays on one CTA: k_pack_chol factors M = C C^T and inverts C (FP64, shared
// memory); then q CTAs form one column each of Lam = C^-T C^-1 and T Lam
// (k_pack_lam), and of Lam (T Lam) with the packed output (k_pack_out).
__global__ void k_pack_chol(int q, const float *Mf, double *Cinv, int *status)
{
    extern __shared__ double sm[];
    double *a = sm;  // C, then C^-1
    if (status_bad(status)) return;
    for (int e = threadIdx.x; e < q * q; e += blockDim.x) {
        const int i = e % q, c = e / q;
        a[e] = 0.5 * ((double)Mf[i + c * q] + (double)Mf[c + i * q]);
    }
    __syncthreads();
    if (!smem_cholesky(a, q)) {
        if (threadIdx.x == 0) atomicOr(status, ST_NOTSPD);
        return;
    }
    smem_tri_inverse(a, q);
    for (int e = threadIdx.x; e < q * q; e += blockDim.x) Cinv[e] = a[e];
}

// block j, thread i: Lam_ij = sum_{k >= max(i, j)} Cinv_ki Cinv_kj, then (T Lam)_ij (T symmetrised)
__global__ void k_pack_lam(int q, const double *Cinv, const float *Tf, double *Lam, double *TL, const int *status)
{
    __shared__ double lj[128];
    if (status_bad(status)) return;
    const int i = threadIdx.x, j = blockIdx.x;
    if (i < q) {
        double s = 0.0;
        for (int k = max(i, j); k < q; ++k) s += Cinv[k + i * q] * Cinv[k + j * q];
        lj[i] = s;
        Lam[i + j * q] = s;
    }
    __syncthreads();
    if (Tf && i < q) {
        double s = 0.0;
        for (int k = 0; k < q; ++k) s += 0.5 * ((double)Tf[i + k * q] + (double)Tf[k + i * q]) * lj[k];
        TL[i + j * q] = s;
    }
}

// block j, thread i: the packed output column j
__global__ void k_pack_out(int q, const double *Lam, const double *TL, int with_t, float *Bw, int *status)
{
    if (status_bad(status)) return;
    const int i = threadIdx.x, j = blockIdx.x;
    if (i >= q) return;
    const double lam = Lam[i + j * q];
    double top = lam;
    if (with_t) {
        double s = 0.0;
        for (int k = 0; k < q; ++k) s += Lam[i + k * q] * TL[k + j * q];  // (Lam T Lam)_ij
        top = 0.5 * (lam + s);
    }
    if (!isfinite(top) || !isfinite(lam)) atomicOr(status, ST_NONFINITE);
    Bw[i + (size_t)j * 2 * q] = (float)top;
    Bw[q + i + (size_t)j * 2 * q] = (float)-lam;
}

void launch_core_pack(cudaStream_t st, int q, const float *Mf, const float *Tf, float *Bw, double *scratch,
                      int *status)
{
    const size_t smem = sizeof(double) * q * q;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_pack_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        attr_set = true;
    }
    double *Cinv = scratch, *Lam = scratch + (size_t)q * q, *TL = scratch + 2 * (size_t)q * q;
    const int tpb = ((q + 31) / 32) * 32;
    rb_count_launch();
    k_pack_chol<<<1, 512, smem, st>>>(q, Mf, Cinv, status);
    rb_count_launch();
    k_pack_lam<<<q, tpb, 0, st>>>(q, Cinv, Tf, Lam, TL, status);
    rb_count_launch();
    k_pack_out<<<q, tpb, 0, st>>>(q, Lam, TL, Tf != nullptr, Bw, status);
}

// ---------------------------------------------------------------------------
// Elementwise helpers
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_set_identity(int n, T *X, int64_t ld, T diag)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i < n) X[i + (int64_t)j * ld] = (i == j) ? diag : T(0);
}

template <typename T>
void launch_set_identity(cudaStream_t st, int n, T *X, int64_t ld, T diag)
{
    dim3 grid(ceil_div(n, 256), n);
    rb_count_launch();
    k_set_identity<T><<<grid, 256, 0, st>>>(n, X, ld, diag);
}
template void launch_set_identity<float>(cudaStream_t, int, float *, int64_t, float);
template void launch_set_identity<double>(cudaStream_t, int, double *, int64_t, double);

// Y (rows x cols, ldy) = alpha * X (ldx), with type conversion.
template <typename Ti, typename To>
__global__ void k_copy2d(int rows, int cols, const Ti *X, int64_t ldx, To *Y, int64_t ldy, double alpha)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i < rows) Y[i + (int64_t)j * ldy] = (To)(alpha * (double)X[i + (int64_t)j * ldx]);
}

template <typename Ti, typename To>
void launch_copy2d(cudaStream_t st, int rows, int cols, const Ti *X, int64_t ldx, To *Y, int64_t ldy, double alpha)
{
    dim3 grid(ceil_div(rows, 256), cols);
    rb_count_launch();
    k_copy2d<Ti, To><<<grid, 256, 0, st>>>(rows, cols, X, ldx, Y, ldy, alpha);
}
template void launch_copy2d<float, float>(cudaStream_t, int, int, const float *, int64_t, float *, int64_t, double);
template void launch_copy2d<double, double>(cudaStream_t, int, int, const double *, int64_t, double *, int64_t,
                                            double);
template void launch_copy2d<float, double>(cudaStream_t, int, int, const float *, int64_t, double *, int64_t,
                                           double);
template void launch_copy2d<double, float>(cudaStream_t, int, int, const double *, int64_t, float *, int64_t,
                                           double);

// diag[i] = A[i + i lda] as double
template <typename T>
__global__ void k_diag(int n, const T *A, int64_t lda, double *d)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) d[i] = (double)A[i + (int64_t)i * lda];
}
template <typename T>
void launch_diag(cudaStream_t st, int n, const T *A, int64_t lda, double *d)
{
    rb_count_launch();
    k_diag<T><<<ceil_div(n, 256), 256, 0, st>>>(n, A, lda, d);
}
template void launch_diag<float>(cudaStream_t, int, const float *, int64_t, double *);
template void launch_diag<double>(cudaStream_t, int, const double *, int64_t, double *);
