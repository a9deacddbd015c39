// sketch.cu -- sketch draws (Sec. 9.3 / Sec. 10 Gaussian S~, Sec. 7 discrete
// coordinate samplings) from the counter-based Philox4x32-10 stream.
#include "kernels.cuh"

// Gaussian sketch, n x q, column-major (ld lds).  Entries (4r + t, j),
// t = 0..3, come from the Philox block with counter (r, j, k, stream) and key
// seed; Box-Muller on word pairs (0,1) and (2,3):
//   rad = sqrt(-2 ln u_a), z_a = rad cos(2 pi u_b), z_b = rad sin(2 pi u_b).
template <typename T>
__global__ void k_gauss_sketch(int n, int q, uint64_t seed, uint64_t stream, uint64_t k, T *S, int64_t lds)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (4 * r >= n || j >= q) return;
    const u32x4 w = philox10((uint32_t)r, (uint32_t)j, (uint32_t)k, (uint32_t)stream, (uint32_t)seed,
                             (uint32_t)(seed >> 32));
    T z[4];
    if constexpr (sizeof(T) == 8) {
        double s, c;
        double rad = sqrt(-2.0 * log(u24d(w.x)));
        sincospi(2.0 * u24d(w.y), &s, &c);
        z[0] = rad * c;
        z[1] = rad * s;
        rad = sqrt(-2.0 * log(u24d(w.z)));
        sincospi(2.0 * u24d(w.w), &s, &c);
        z[2] = rad * c;
        z[3] = rad * s;
    } else {
        float s, c;
        float rad = sqrtf(-2.0f * logf(u24f(w.x)));
        sincospif(2.0f * u24f(w.y), &s, &c);
        z[0] = rad * c;
        z[1] = rad * s;
        rad = sqrtf(-2.0f * logf(u24f(w.z)));
        sincospif(2.0f * u24f(w.w), &s, &c);
        z[2] = rad * c;
        z[3] = rad * s;
    }
    T *col = S + (int64_t)j * lds;
#pragma unroll
    for (int t = 0; t < 4; ++t)
        if (4 * r + t < n) col[4 * r + t] = z[t];
}

template <typename T>
void launch_gauss_sketch(cudaStream_t st, int n, int q, uint64_t seed, uint64_t stream, uint64_t k, T *S,
                         int64_t lds)
{
    dim3 grid(ceil_div((n + 3) / 4, 128), q);
    rb_count_launch();
    k_gauss_sketch<T><<<grid, 128, 0, st>>>(n, q, seed, stream, k, S, lds);
}
template void launch_gauss_sketch<float>(cudaStream_t, int, int, uint64_t, uint64_t, uint64_t, float *, int64_t);
template void launch_gauss_sketch<double>(cudaStream_t, int, int, uint64_t, uint64_t, uint64_t, double *, int64_t);

// Trace-weighted coordinate block: one 64-bit draw r from counter
// (0, TAG_COORD, k, stream), t = floor(r W / 2^64) with W = P[nb] the total
// integer weight, block b with P[b] <= t < P[b+1].  Writes (first, size).
__global__ void k_coord_trace_draw(int n, int q, int nb, const uint64_t *P, uint64_t seed, uint64_t stream,
                                   uint64_t k, int *blk)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const u32x4 w = philox10(0u, TAG_COORD, (uint32_t)k, (uint32_t)stream, (uint32_t)seed, (uint32_t)(seed >> 32));
    const uint64_t r = (uint64_t)w.x | ((uint64_t)w.y << 32);
    const uint64_t t = __umul64hi(r, P[nb]);
    int lo = 0, hi = nb - 1;  // largest b with P[b] <= t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P[mid] <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    blk[0] = lo * q;
    blk[1] = ((lo + 1) * q <= n) ? q : n - lo * q;
}

void launch_coord_trace_draw(cudaStream_t st, int n, int q, int nb, const uint64_t *P, uint64_t seed,
                             uint64_t stream, uint64_t k, int *blk)
{
    rb_count_launch();
    k_coord_trace_draw<<<1, 32, 0, st>>>(n, q, nb, P, seed, stream, k, blk);
}

// q distinct coordinates of [0, n), uniform: Floyd's algorithm with draw i
// from counter (i, TAG_COORD, k, stream), d = floor(x (t + 1) / 2^32) for
// t = n - q + i; sorted ascending.  One thread (q <= 128).
__global__ void k_floyd_draw(int n, int q, uint64_t seed, uint64_t stream, uint64_t k, int *idx)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = 0; i < q; ++i) {
        const uint32_t t = (uint32_t)(n - q + i);
        const u32x4 w = philox10((uint32_t)i, TAG_COORD, (uint32_t)k, (uint32_t)stream, (uint32_t)seed,
                                 (uint32_t)(seed >> 32));
        const int d = (int)(((uint64_t)w.x * (uint64_t)(t + 1u)) >> 32);
        bool seen = false;
        for (int a = 0; a < i; ++a) seen |= (idx[a] == d);
        idx[i] = seen ? (int)t : d;
    }
    for (int i = 1; i < q; ++i) {  // insertion sort
        const int v = idx[i];
        int a = i - 1;
        while (a >= 0 && idx[a] > v) {
            idx[a + 1] = idx[a];
            --a;
        }
        idx[a + 1] = v;
    }
}

void launch_floyd_draw(cudaStream_t st, int n, int q, uint64_t seed, uint64_t stream, uint64_t k, int *idx)
{
    rb_count_launch();
    k_floyd_draw<<<1, 32, 0, st>>>(n, q, seed, stream, k, idx);
}

// S~ = I[:, idx] as an explicit n x q 0/1 matrix (AdaRBFGS_cols).
template <typename T>
__global__ void k_coord_matrix(int n, int q, const int *idx, T *S, int64_t lds)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (i >= n) return;
    S[i + (int64_t)c * lds] = (i == idx[c]) ? T(1) : T(0);
}

template <typename T>
void launch_coord_matrix(cudaStream_t st, int n, int q, const int *idx, T *S, int64_t lds)
{
    dim3 grid(ceil_div(n, 256), q);
    rb_count_launch();
    k_coord_matrix<T><<<grid, 256, 0, st>>>(n, q, idx, S, lds);
}
template void launch_coord_matrix<float>(cudaStream_t, int, int, const int *, float *, int64_t);
template void launch_coord_matrix<double>(cudaStream_t, int, int, const int *, double *, int64_t);

// I[:, C] for a contiguous block blk = {first, size}; zero columns c >= size.
template <typename T>
__global__ void k_block_matrix(int n, int q, const int *blk, T *S, int64_t lds)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (i >= n) return;
    S[i + (int64_t)c * lds] = (c < blk[1] && i == blk[0] + c) ? T(1) : T(0);
}

template <typename T>
void launch_block_matrix(cudaStream_t st, int n, int q, const int *blk, T *S, int64_t lds)
{
    dim3 grid(ceil_div(n, 256), q);
    rb_count_launch();
    k_block_matrix<T><<<grid, 256, 0, st>>>(n, q, blk, S, lds);
}
template void launch_block_matrix<float>(cudaStream_t, int, int, const int *, float *, int64_t);
template void launch_block_matrix<double>(cudaStream_t, int, int, const int *, double *, int64_t);
