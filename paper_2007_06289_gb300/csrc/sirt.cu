// Algebraic reconstruction on the fast Hough operators (the FHT-based iterative method the
// paper points to in Sec. 4.4), in its simultaneous form:
//     f <- f + lam C^-1 A^T (R^-1 (b - A f)),   R = A 1,  C = A^T 1,
// A the dyadic line sums of an image (the transposed back projection, adjoint.cu) and A^T
// the back projection of a linogram (the two Hough passes, fht.cu).  The residual
// (b - A f) R^-1 is formed by the projection's last launch as it writes A f (adjoint.cu).
// This file holds the update step, the fill and reciprocal that make R^-1 and C^-1, the
// conversion of a sinogram into Hough-space data (the sinogram sampled at the linogram
// points, Eq. 14-15, divided by the path length per row sqrt(1 + sigma^2), since a dyadic
// line visits one pixel per row), and the opposite resampling, which turns the line sums of
// the fast Hough projection (Eq. 17) into a (theta, r) sinogram: a fast Radon transform.
#include "fbp_internal.h"

namespace fbp {
namespace {

constexpr int kSirtThreads = 256;

// value of detector bin j of a sinogram row, zero outside [0, M) (and, in the bounds-checked
// build, outside the sinogram buffer)
__device__ __forceinline__ float bin_or_zero(const Span& sp, const float* row, int M, int j)
{
    return (j >= 0 && j < M) ? ld_in(sp, row + j) : 0.0f;
}

// b[q][i][c] = hw.x * lerp(row k0) + hw.y * lerp(row k0 + 1, or row 0 mirrored past the last
// angle), hw = ((1 - ft), ft) / sqrt(1 + sigma^2); positions as in the forward resampling.
__global__ void __launch_bounds__(kSirtThreads)
hough_data_kernel(const float* __restrict__ sino, float* __restrict__ lin,
                  const RowGeom* __restrict__ geom, const float2* __restrict__ hw, int N, int K,
                  int M, int count, int* status)
{
    const int W = 2 * N;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int qi = blockIdx.y;                  // q * N + i
    const int s = blockIdx.z;
    if (c >= W) return;
    const Span sp{sino, (long long)count * K * M, status};
    const long long o = ((long long)s * 4 * N + qi) * W + c;
    if (!in_bounds(status, o, (long long)count * 4 * N * W)) return;
    const RowGeom gm = geom[qi];
    if (!row_geom_valid(gm, K)) {               // rejected geometry row: zeros
        if (c == 0) flag_status(status, (int)FBP_ERR_INTERNAL);
        lin[o] = 0.0f;
        return;
    }
    const float2 w = hw[qi];
    const float* ps = sino + (size_t)s * K * M;
    const long long m = gm.b_fx + gm.a_fx * (long long)c;
    const int j = (int)(m >> kFixBits);
    const float f = __uint2float_rn((unsigned)m) * 0x1p-32f;
    const float* ra = ps + (size_t)gm.k0 * M;
    const float a0 = bin_or_zero(sp, ra, M, j), a1 = bin_or_zero(sp, ra, M, j + 1);
    const float va = fmaf(f, a1 - a0, a0);
    float vb;
    if (!gm.wrap) {
        const float* rb = ra + M;
        const float b0 = bin_or_zero(sp, rb, M, j), b1 = bin_or_zero(sp, rb, M, j + 1);
        vb = fmaf(f, b1 - b0, b0);
    } else {
        const long long mm = ((long long)(M - 1) << kFixBits) - m;
        const int jm = (int)(mm >> kFixBits);
        const float fm = __uint2float_rn((unsigned)mm) * 0x1p-32f;
        const float b0 = bin_or_zero(sp, ps, M, jm), b1 = bin_or_zero(sp, ps, M, jm + 1);
        vb = fmaf(fm, b1 - b0, b0);
    }
    lin[o] = fmaf(w.y, vb, w.x * va);
}

// Fast Radon transform: sinogram row k from the dyadic line sums H of its line class, the
// two linogram rows around its slope read at the column of detector offset r_m (linear in
// the column, zero outside [0, 2N)), mixed (1 - t, t), times the path length per row.
__global__ void __launch_bounds__(kSirtThreads)
radon_kernel(const float* __restrict__ lin, float* __restrict__ sino,
             const RadonRow* __restrict__ rows, int N, int K, int M, int count, int* status)
{
    const int W = 2 * N;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    const int s = blockIdx.z;
    if (m >= M) return;
    const long long o = ((long long)s * K + k) * M + m;
    if (!in_bounds(status, o, (long long)count * K * M)) return;
    const RadonRow e = rows[k];
    const Span sl{lin, (long long)count * 4 * N * W, status};
    const float* h = lin + (((size_t)s * 4 + e.q) * N + e.i0) * W;
    float v[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const long long cf = e.b_fx[j] + e.a_fx[j] * (long long)m;
        const int c = (int)(cf >> kFixBits);
        const float f = __uint2float_rn((unsigned)cf) * 0x1p-32f;
        const float* row = h + (size_t)j * W;
        const float h0 = (c >= 0 && c < W) ? ld_in(sl, row + c) : 0.0f;
        const float h1 = (c + 1 >= 0 && c + 1 < W) ? ld_in(sl, row + c + 1) : 0.0f;
        v[j] = fmaf(f, h1, (1.0f - f) * h0);
    }
    sino[o] = fmaf(e.t, v[1], (1.0f - e.t) * v[0]) * e.scale;
}

// f = f + lam * cinv * t
__global__ void __launch_bounds__(kSirtThreads)
sirt_update_kernel(float4* __restrict__ f, const float4* __restrict__ t,
                   const float4* __restrict__ cinv, float lam, size_t per_slice4, size_t total4)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total4;
         i += (size_t)gridDim.x * blockDim.x) {
        const float4 ff = f[i], tt = t[i], w = cinv[i % per_slice4];
        f[i] = make_float4(ff.x + lam * w.x * tt.x, ff.y + lam * w.y * tt.y,
                           ff.z + lam * w.z * tt.z, ff.w + lam * w.w * tt.w);
    }
}

__global__ void __launch_bounds__(kSirtThreads)
fill_kernel(float* __restrict__ x, float v, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        x[i] = v;
}

// x = 1 / x where x > 0, else 0
__global__ void __launch_bounds__(kSirtThreads)
recip_kernel(float* __restrict__ x, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        x[i] = x[i] > 0.0f ? 1.0f / x[i] : 0.0f;
}

int stream_grid(size_t n)
{
    const size_t blocks = (n + kSirtThreads - 1) / kSirtThreads;
    return (int)(blocks < 4096 ? (blocks > 0 ? blocks : 1) : 4096);
}

}  // namespace

cudaError_t launch_hough_data(const fbp_plan_s* p, const float* sino, float* lin, int count,
                              cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    const dim3 grid((2 * p->N + kSirtThreads - 1) / kSirtThreads, 4 * p->N, count);
    hough_data_kernel<<<grid, kSirtThreads, 0, st>>>(sino, lin, p->d_geom, p->d_hough_w, p->N,
                                                     p->K, p->M, count, p->d_status);
    return cudaGetLastError();
}

cudaError_t launch_radon(const fbp_plan_s* p, const float* lin, float* sino, int count,
                         cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    const dim3 grid((p->M + kSirtThreads - 1) / kSirtThreads, p->K, count);
    radon_kernel<<<grid, kSirtThreads, 0, st>>>(lin, sino, p->d_radon, p->N, p->K, p->M, count,
                                                p->d_status);
    return cudaGetLastError();
}

cudaError_t launch_sirt_update(float* f, const float* t, const float* cinv, float lam,
                               size_t per_slice, int count, cudaStream_t st)
{
    const size_t total4 = per_slice / 4 * count;
    sirt_update_kernel<<<stream_grid(total4), kSirtThreads, 0, st>>>(
        reinterpret_cast<float4*>(f), reinterpret_cast<const float4*>(t),
        reinterpret_cast<const float4*>(cinv), lam, per_slice / 4, total4);
    return cudaGetLastError();
}

cudaError_t launch_fill(float* x, float v, size_t n, cudaStream_t st)
{
    fill_kernel<<<stream_grid(n), kSirtThreads, 0, st>>>(x, v, n);
    return cudaGetLastError();
}

cudaError_t launch_recip(float* x, size_t n, cudaStream_t st)
{
    recip_kernel<<<stream_grid(n), kSirtThreads, 0, st>>>(x, n);
    return cudaGetLastError();
}

}  // namespace fbp
