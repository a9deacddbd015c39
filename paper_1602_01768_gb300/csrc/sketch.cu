// sketch.cu -- sketch draws (Sec. 9.3 / Sec. 10 Gaussian S~, Sec. 7 discrete
// coordinate samplings) from the counter-based Philox4x32-10 stream.
#include "kernels.cuh"

// Gaussian sketch entries are defined by binary32 arithmetic in a fixed
// order -- every step a correctly rounded IEEE operation (the _rn intrinsics
// keep the compiler from contracting or reordering), polynomials by fmaf in
// Horner order -- and then rounded to the nearest TF32 value, so the sketch is
// reproducible bit for bit on any IEEE machine and exact in one tensor-core
// pass.  The elementary functions come from their Taylor series:
//
// ln u, u in (0, 1]: u = m 2^e, m in [sqrt(1/2), sqrt(2)); ln m = 2 atanh(s),
// s = (m - 1)/(m + 1), atanh(s) = s + s^3/3 + s^5/5 + s^7/7 + s^9/9;
// ln u = e ln2_hi + (e ln2_lo + ln m), ln2_hi with 16 significant bits.
__device__ __forceinline__ float bm_log(float u)
{
    const uint32_t b = __float_as_uint(u);
    int e = (int)((b >> 23) & 0xffu) - 127;
    float m = __uint_as_float((b & 0x007fffffu) | 0x3f800000u);  // [1, 2)
    if (m > 1.41421354f) {
        m = __fmul_rn(m, 0.5f);
        e += 1;
    }
    const float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float s2 = __fmul_rn(s, s);
    float p = __fmaf_rn(s2, 0.111111112f, 0.142857149f);
    p = __fmaf_rn(s2, p, 0.200000003f);
    p = __fmaf_rn(s2, p, 0.333333343f);
    const float at = __fmaf_rn(__fmul_rn(s, s2), p, s);
    const float lm = __fmul_rn(2.0f, at);
    const float t = __fmaf_rn((float)e, 1.42860676e-06f, lm);
    return __fadd_rn(__fmul_rn((float)e, 0.693145751953125f), t);
}

// sin(pi x), cos(pi x), x in [0, 2]: k = nearest integer to 2x, r = x - k/2
// in [-1/4, 1/4] (exact), t = pi r; Taylor polynomials of sin t (to t^11) and
// cos t (to t^12); the quarter turn k mod 4 selects and signs them.
__device__ __forceinline__ void bm_sincospi(float x, float *sp, float *cp)
{
    const float k = rintf(__fmul_rn(2.0f, x));
    const float r = __fsub_rn(x, __fmul_rn(0.5f, k));
    const float t = __fmul_rn(r, 3.14159274f);
    const float t2 = __fmul_rn(t, t);
    float ps = __fmaf_rn(t2, -2.50521079e-08f, 2.75573188e-06f);
    ps = __fmaf_rn(t2, ps, -1.98412701e-04f);
    ps = __fmaf_rn(t2, ps, 8.33333377e-03f);
    ps = __fmaf_rn(t2, ps, -0.166666672f);
    const float sn = __fmaf_rn(__fmul_rn(t, t2), ps, t);
    float pc = __fmaf_rn(t2, 2.08767570e-09f, -2.75573188e-07f);
    pc = __fmaf_rn(t2, pc, 2.48015876e-05f);
    pc = __fmaf_rn(t2, pc, -1.38888892e-03f);
    pc = __fmaf_rn(t2, pc, 4.16666679e-02f);
    pc = __fmaf_rn(t2, pc, -0.5f);
    const float cs = __fmaf_rn(t2, pc, 1.0f);
    switch ((int)k & 3) {
    case 0: *sp = sn; *cp = cs; break;
    case 1: *sp = cs; *cp = -sn; break;
    case 2: *sp = -sn; *cp = -cs; break;
    default: *sp = -cs; *cp = sn; break;
    }
}

// nearest TF32 value (10 stored fraction bits), ties to even
__device__ __forceinline__ float to_tf32_rne(float z)
{
    uint32_t b = __float_as_uint(z);
    const uint32_t r = b & 0x1fffu;
    b &= ~0x1fffu;
    if (r > 0x1000u || (r == 0x1000u && (b & 0x2000u))) b += 0x2000u;
    return __uint_as_float(b);
}

// binary32 uniform ((x >> 8) + 1/2) 2^-24 (above 1/2 the sum rounds to even)
__device__ __forceinline__ float bm_uniform(uint32_t x) { return __fmul_rn(__fadd_rn((float)(x >> 8), 0.5f), 5.96046448e-08f); }

// Gaussian sketch, n x q, column-major (ld lds).  Entries (4r + t, j),
// t = 0..3, come from the Philox block with counter (r, j, k, stream) and key
// seed; Box-Muller on word pairs (0,1) and (2,3):
//   rad = sqrt(-2 ln u_a), z_a = rad cos(2 pi u_b), z_b = rad sin(2 pi u_b),
// each entry rounded to TF32 (stored as T).
template <typename T>
__global__ void k_gauss_sketch(int n, int q, uint64_t seed, uint64_t stream, uint64_t k, T *S, int64_t lds)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (4 * r >= n || j >= q) return;
    const u32x4 w = philox10((uint32_t)r, (uint32_t)j, (uint32_t)k, (uint32_t)stream, (uint32_t)seed,
                             (uint32_t)(seed >> 32));
    const uint32_t wv[4] = {w.x, w.y, w.z, w.w};
    T z[4];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const float rad = __fsqrt_rn(__fmul_rn(-2.0f, bm_log(bm_uniform(wv[2 * p]))));
        float sn, cs;
        bm_sincospi(__fmul_rn(2.0f, bm_uniform(wv[2 * p + 1])), &sn, &cs);
        z[2 * p] = (T)to_tf32_rne(__fmul_rn(rad, cs));
        z[2 * p + 1] = (T)to_tf32_rne(__fmul_rn(rad, sn));
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
