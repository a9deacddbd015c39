// aux.cu -- residual monitor, coordinate-block helpers of RBFGS, and the
// reductions of the comparison methods.
#include "kernels.cuh"

// ---------------------------------------------------------------------------
// Residual ||I - X A||_F^2 pieces.  Z (n x m) holds X A e_{J[c]} in column c;
// each block sums (delta_{i, J[c]} - Z_ic)^2 over its rows in FP64 and writes
// a partial; the partials are summed in fixed order.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_resid_partial(int n, int m, const T *Z, int64_t ldz, const int *J, double *part)
{
    __shared__ double red[256];
    const int c = blockIdx.y;
    const int jc = J ? J[c] : c;
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double e = ((i == jc) ? 1.0 : 0.0) - (double)Z[i + (int64_t)c * ldz];
        s += e * e;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x + (size_t)blockIdx.y * gridDim.x] = red[0];
}

__global__ void k_sum_fixed(int cnt, const double *part, double *out)
{
    __shared__ double red[256];
    double s = 0.0;
    for (int e = threadIdx.x; e < cnt; e += 256) s += part[e];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

template <typename T>
void launch_resid_sumsq(cudaStream_t st, int n, int m, const T *Z, int64_t ldz, const int *J, double *part,
                        double *out)
{
    const int bx = min(ceil_div(n, 256), 32);
    dim3 grid(bx, m);
    rb_count_launch();
    k_resid_partial<T><<<grid, 256, 0, st>>>(n, m, Z, ldz, J, part);
    rb_count_launch();
    k_sum_fixed<<<1, 256, 0, st>>>(bx * m, part, out);
}
template void launch_resid_sumsq<float>(cudaStream_t, int, int, const float *, int64_t, const int *, double *,
                                        double *);
template void launch_resid_sumsq<double>(cudaStream_t, int, int, const double *, int64_t, const int *, double *,
                                         double *);

// Y[:, c] = A[:, J[c]]
template <typename T>
__global__ void k_gather_cols(int n, int m, const T *A, int64_t lda, const int *J, T *Y, int64_t ldy)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (i < n) Y[i + (int64_t)c * ldy] = A[i + (int64_t)J[c] * lda];
}
template <typename T>
void launch_gather_cols(cudaStream_t st, int n, int m, const T *A, int64_t lda, const int *J, T *Y, int64_t ldy)
{
    dim3 grid(ceil_div(n, 256), m);
    rb_count_launch();
    k_gather_cols<T><<<grid, 256, 0, st>>>(n, m, A, lda, J, Y, ldy);
}
template void launch_gather_cols<float>(cudaStream_t, int, int, const float *, int64_t, const int *, float *,
                                        int64_t);
template void launch_gather_cols<double>(cudaStream_t, int, int, const double *, int64_t, const int *, double *,
                                         int64_t);

// ---------------------------------------------------------------------------
// RBFGS with a coordinate block C = [first, first + size) (device-resident,
// blk = {first, size}); q is the block width the buffers are sized for.
//   G = A[:, C] (zero columns beyond size); Mpad = A[C, C] padded with I so
//   its Cholesky exists; S B1 adds B1 to rows C of W; the update X += S W^T +
//   W S^T touches rows and columns C only.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_coord_gather(int n, int q, const T *A, int64_t lda, const int *blk, T *G, int64_t ldg,
                               double *Mpad, const int *status)
{
    if (status_bad(status)) return;
    const int first = blk[0], size = blk[1];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (i >= n) return;
    const T v = (c < size) ? A[i + (int64_t)(first + c) * lda] : T(0);
    G[i + (int64_t)c * ldg] = v;
    const int r = i - first;
    if (r >= 0 && r < q) {
        double mv;
        if (r < size && c < size)
            mv = (double)v;
        else
            mv = (r == c) ? 1.0 : 0.0;
        Mpad[r + c * q] = mv;
    }
}

// Rows of Mpad with first + r >= n (ragged last block) are not touched by
// k_coord_gather; fill them here.
__global__ void k_coord_pad_rows(int n, int q, const int *blk, double *Mpad, const int *status)
{
    if (status_bad(status)) return;
    const int first = blk[0];
    const int r = threadIdx.x + blockIdx.x * blockDim.x;
    const int c = blockIdx.y;
    if (r < q && first + r >= n) Mpad[r + c * q] = (r == c) ? 1.0 : 0.0;
}

template <typename T>
void launch_coord_gather(cudaStream_t st, int n, int q, const T *A, int64_t lda, const int *blk, T *G, int64_t ldg,
                         double *Mpad, const int *status)
{
    dim3 grid(ceil_div(n, 256), q);
    rb_count_launch();
    k_coord_gather<T><<<grid, 256, 0, st>>>(n, q, A, lda, blk, G, ldg, Mpad, status);
    dim3 g2(ceil_div(q, 128), q);
    rb_count_launch();
    k_coord_pad_rows<<<g2, 128, 0, st>>>(n, q, blk, Mpad, status);
}
template void launch_coord_gather<float>(cudaStream_t, int, int, const float *, int64_t, const int *, float *,
                                         int64_t, double *, const int *);
template void launch_coord_gather<double>(cudaStream_t, int, int, const double *, int64_t, const int *, double *,
                                          int64_t, double *, const int *);

// W[first + r, c] += B1[r, c] for r, c < size (the S B1 term with S = I[:, C]).
template <typename T>
__global__ void k_coord_add_b1(int q, const int *blk, const T *B1, T *W, int64_t ldw, const int *status)
{
    if (status_bad(status)) return;
    const int first = blk[0], size = blk[1];
    const int r = threadIdx.x, c = blockIdx.x;
    if (r < size && c < size) W[first + r + (int64_t)c * ldw] += B1[r + c * q];
}

template <typename T>
void launch_coord_add_b1(cudaStream_t st, int q, const int *blk, const T *B1, T *W, int64_t ldw, const int *status)
{
    rb_count_launch();
    k_coord_add_b1<T><<<q, q, 0, st>>>(q, blk, B1, W, ldw, status);
}
template void launch_coord_add_b1<float>(cudaStream_t, int, const int *, const float *, float *, int64_t,
                                         const int *);
template void launch_coord_add_b1<double>(cudaStream_t, int, const int *, const double *, double *, int64_t,
                                          const int *);

// X += S W^T + W S^T with S = I[:, C]:
//   columns first + c (all rows i): X[i, f+c] += W[i, c] + [i in C] W[f+c, i-f]
//   rows first + r, columns j not in C: X[f+r, j] += W[j, r]
template <typename T>
__global__ void k_coord_update_cols(int n, int q, const int *blk, const T *W, int64_t ldw, T *X, int64_t ldx,
                                    const int *status)
{
    if (status_bad(status)) return;
    const int first = blk[0], size = blk[1];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (i >= n || c >= size) return;
    T d = W[i + (int64_t)c * ldw];
    const int r = i - first;
    if (r >= 0 && r < size) d += W[first + c + (int64_t)r * ldw];
    X[i + (int64_t)(first + c) * ldx] += d;
}

template <typename T>
__global__ void k_coord_update_rows(int n, int q, const int *blk, const T *W, int64_t ldw, T *X, int64_t ldx,
                                    const int *status)
{
    if (status_bad(status)) return;
    const int first = blk[0], size = blk[1];
    const int r = threadIdx.x % 32;
    const int j = blockIdx.x * 8 + threadIdx.x / 32;
    if (j >= n || (j >= first && j < first + size)) return;
    for (int rr = r; rr < size; rr += 32) X[first + rr + (int64_t)j * ldx] += W[j + (int64_t)rr * ldw];
}

template <typename T>
void launch_coord_update(cudaStream_t st, int n, int q, const int *blk, const T *W, int64_t ldw, T *X, int64_t ldx,
                         const int *status)
{
    dim3 g1(ceil_div(n, 256), q);
    rb_count_launch();
    k_coord_update_cols<T><<<g1, 256, 0, st>>>(n, q, blk, W, ldw, X, ldx, status);
    rb_count_launch();
    k_coord_update_rows<T><<<ceil_div(n, 8), 256, 0, st>>>(n, q, blk, W, ldw, X, ldx, status);
}
template void launch_coord_update<float>(cudaStream_t, int, int, const int *, const float *, int64_t, float *,
                                         int64_t, const int *);
template void launch_coord_update<double>(cudaStream_t, int, int, const int *, const double *, int64_t, double *,
                                          int64_t, const int *);

// ---------------------------------------------------------------------------
// Reductions of the comparison methods (FP64 accumulation).
// ---------------------------------------------------------------------------

// out = {sum R .* Q, sum Q .* Q} over an n x n pair: partials per block,
// then summed in fixed order by k_sum2_fixed.
template <typename T>
__global__ void k_mr_dots_partial(int n, const T *P, int64_t ldp, const T *Q, int64_t ldq, double *part)
{
    __shared__ double r0[256], r1[256];
    double a = 0.0, b = 0.0;
    const int64_t total = (int64_t)n * n;
    for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < total; e += (int64_t)gridDim.x * 256) {
        const int i = (int)(e % n), j = (int)(e / n);
        const double r = (double)P[i + (int64_t)j * ldp];
        const double qv = (double)Q[i + (int64_t)j * ldq];
        a += r * qv;
        b += qv * qv;
    }
    r0[threadIdx.x] = a;
    r1[threadIdx.x] = b;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            r0[threadIdx.x] += r0[threadIdx.x + w];
            r1[threadIdx.x] += r1[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = r0[0];
        part[2 * blockIdx.x + 1] = r1[0];
    }
}

__global__ void k_sum2_fixed(int cnt, const double *part, double *out)
{
    if (threadIdx.x != 0) return;
    double a = 0.0, b = 0.0;
    for (int e = 0; e < cnt; ++e) {
        a += part[2 * e];
        b += part[2 * e + 1];
    }
    out[0] = a;
    out[1] = b;
}

template <typename T>
void launch_mr_dots(cudaStream_t st, int n, const T *P, int64_t ldp, const T *Q, int64_t ldq, double *part,
                    double *out)
{
    const int blocks = 512;
    rb_count_launch();
    k_mr_dots_partial<T><<<blocks, 256, 0, st>>>(n, P, ldp, Q, ldq, part);
    rb_count_launch();
    k_sum2_fixed<<<1, 32, 0, st>>>(blocks, part, out);
}
template void launch_mr_dots<float>(cudaStream_t, int, const float *, int64_t, const float *, int64_t, double *,
                                    double *);
template void launch_mr_dots<double>(cudaStream_t, int, const double *, int64_t, const double *, int64_t,
                                     double *, double *);

// R = I - P in place (P n x n).
template <typename T>
__global__ void k_i_minus(int n, T *P, int64_t ld)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i < n) {
        T *p = P + i + (int64_t)j * ld;
        *p = ((i == j) ? T(1) : T(0)) - *p;
    }
}
template <typename T>
void launch_i_minus(cudaStream_t st, int n, T *P, int64_t ld)
{
    dim3 grid(ceil_div(n, 256), n);
    rb_count_launch();
    k_i_minus<T><<<grid, 256, 0, st>>>(n, P, ld);
}
template void launch_i_minus<float>(cudaStream_t, int, float *, int64_t);
template void launch_i_minus<double>(cudaStream_t, int, double *, int64_t);

// X += (num/den) D, alpha read from device (dots = {num, den}).
template <typename T>
__global__ void k_axpy_dev(int n, const double *dots, const T *D, int64_t ldd, T *X, int64_t ldx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    const double den = dots[1];
    const double alpha = den > 0.0 ? dots[0] / den : 0.0;
    if (i < n) X[i + (int64_t)j * ldx] += (T)(alpha * (double)D[i + (int64_t)j * ldd]);
}
template <typename T>
void launch_axpy_dev(cudaStream_t st, int n, const double *dots, const T *D, int64_t ldd, T *X, int64_t ldx)
{
    dim3 grid(ceil_div(n, 256), n);
    rb_count_launch();
    k_axpy_dev<T><<<grid, 256, 0, st>>>(n, dots, D, ldd, X, ldx);
}
template void launch_axpy_dev<float>(cudaStream_t, int, const double *, const float *, int64_t, float *, int64_t);
template void launch_axpy_dev<double>(cudaStream_t, int, const double *, const double *, int64_t, double *,
                                      int64_t);

// Power iteration step: w = A v (v, w length n), norm^2 of w into part sums.
template <typename T>
__global__ void k_gemv_sq(int n, const T *A, int64_t lda, const double *v, double *w)
{
    // one warp per row i (A symmetric: row i = column i, contiguous)
    const int i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    double s = 0.0;
    for (int k = lane; k < n; k += 32) s += (double)A[k + (int64_t)i * lda] * v[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) w[i] = s;
}

__global__ void k_normalize(int n, const double *w, double *v, double *sigma)
{
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) s += w[i] * w[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    const double nrm = sqrt(red[0]);
    for (int i = threadIdx.x; i < n; i += 256) v[i] = w[i] / nrm;
    if (threadIdx.x == 0) *sigma = nrm;
}

__global__ void k_fill(int n, double *v, double val)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = val;
}

template <typename T>
void launch_power_iteration(cudaStream_t st, int n, const T *A, int64_t lda, int iters, double *v, double *w,
                            double *sigma)
{
    rb_count_launch();
    k_fill<<<ceil_div(n, 256), 256, 0, st>>>(n, v, 1.0 / sqrt((double)n));
    for (int it = 0; it < iters; ++it) {
        rb_count_launch();
        k_gemv_sq<T><<<ceil_div(n, 8), 256, 0, st>>>(n, A, lda, v, w);
        rb_count_launch();
        k_normalize<<<1, 256, 0, st>>>(n, w, v, sigma);
    }
}
template void launch_power_iteration<float>(cudaStream_t, int, const float *, int64_t, int, double *, double *,
                                            double *);
template void launch_power_iteration<double>(cudaStream_t, int, const double *, int64_t, int, double *, double *,
                                             double *);

// ---------------------------------------------------------------------------
// Approximate inverse preconditioning, Eq. (BFGSas), with a coordinate block
// C = {first, .., first + size - 1}: S^T = I[C, :], so Lambda S^T adds the
// columns of Lambda into columns C of V, and X += S V changes rows C only.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_aip_add_lam(int q, const int *blk, const T *Lam, T *V, int64_t ldv, const int *status)
{
    if (status_bad(status)) return;
    const int first = blk[0], size = blk[1];
    const int c = threadIdx.x, j = blockIdx.x;
    if (c < q && j < size) V[c + (int64_t)(first + j) * ldv] += Lam[c + (int64_t)j * q];
}

template <typename T>
__global__ void k_aip_update_rows(int n, const int *blk, const T *V, int64_t ldv, T *X, int64_t ldx,
                                  const int *status)
{
    if (status_bad(status)) return;
    const int first = blk[0], size = blk[1];
    const int j = blockIdx.x * blockDim.y + threadIdx.y, i = threadIdx.x;
    if (j < n && i < size) X[(first + i) + (int64_t)j * ldx] += V[i + (int64_t)j * ldv];
}

template <typename T>
void launch_aip_coord(cudaStream_t st, int n, int q, const int *blk, const T *Lam, T *V, int64_t ldv, T *X,
                      int64_t ldx, const int *status)
{
    rb_count_launch();
    k_aip_add_lam<T><<<q, std::max(32, ((q + 31) / 32) * 32), 0, st>>>(q, blk, Lam, V, ldv, status);
    const int ty = std::max(1, 256 / std::max(1, ((q + 31) / 32) * 32));
    dim3 blkdim(((q + 31) / 32) * 32, ty);
    rb_count_launch();
    k_aip_update_rows<T><<<(n + ty - 1) / ty, blkdim, 0, st>>>(n, blk, V, ldv, X, ldx, status);
}
template void launch_aip_coord<float>(cudaStream_t, int, int, const int *, const float *, float *, int64_t, float *,
                                      int64_t, const int *);
template void launch_aip_coord<double>(cudaStream_t, int, int, const int *, const double *, double *, int64_t,
                                       double *, int64_t, const int *);


// out[off + c + i rp] = X[i + c ldx]: thread (i, c), coalesced reads along i.
__global__ void k_rows_from_cols(int n, int q, const float *X, int64_t ldx, float *out, int rp, int off)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, c = blockIdx.y;
    if (i < n) out[off + c + (int64_t)i * rp] = X[i + (int64_t)c * ldx];
}

void launch_rows_from_cols(cudaStream_t st, int n, int q, const float *X, int64_t ldx, float *out, int rp, int off)
{
    rb_count_launch();
    k_rows_from_cols<<<dim3((n + 255) / 256, q), 256, 0, st>>>(n, q, X, ldx, out, rp, off);
}
