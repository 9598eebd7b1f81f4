// Adjoints of the back projection and of the resampling: the transposed operators that carry
// an image-space gradient back to the linogram and to the filtered sinogram (the
// differentiable form of Sec. 4; the filter's adjoint is the filter itself, Eq. 12-13 being
// symmetric).
//
// Back projection, transposed.  Per quarter the forward map is F[tau][u] = sum_i
// L[i][u + d_tau(i)] evaluated by log2 N stages of pair additions (Sec. 4.4-4.5); its
// transpose runs the stages backwards, each stage transposed:
//     A_{k-1}[2b][t][u]   = A_k[b][2t][u] + A_k[b][2t+1][u]
//     A_{k-1}[2b+1][t][v] = A_k[b][2t][v - t] + A_k[b][2t+1][v - t - 1]
// (columns below 0 read as zero), starting from the quarter gradients of Eq. 22's index maps
// and ending with L-bar[i][c] = A_0[i][0][c].  One launch per stage over all slices and
// quarters, ping-ponging between two [count][4][N][2N] buffers; every output element is
// one fixed float32 sum, so the result is reproducible bit for bit.
//
// Resampling, transposed.  Each linogram sample is w0 * lerp(row k0) + w1 * lerp(row k1)
// (Eq. 14-15 with the float32 weights the forward kernels use); its transpose adds the
// sample's gradient times the four bilinear weights into the sinogram gradient with
// atomics (so the summation order, and the last bits, vary from run to run).
#include "fbp_internal.h"

namespace fbp {
namespace {

constexpr int kAdjThreads = 256;

// Quarter gradients (transpose of Eq. 22's sum): g[N][N] -> A_n[4][N][W], zero for u >= N.
//   v-: g[tau][u]   v+: g[tau][N-1-u]   h-: g[u][tau]   h+: g[N-1-u][tau]
__global__ void __launch_bounds__(kAdjThreads)
adj_quarters_kernel(const float* __restrict__ g, float* __restrict__ A, int N, int W)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    const int tau = blockIdx.y;
    const int sq = blockIdx.z;                  // slice * 4 + quarter
    const int q = sq & 3;
    if (u >= W) return;
    const float* gs = g + (size_t)(sq >> 2) * N * N;
    float v = 0.0f;
    if (u < N) {
        switch (q) {
            case 0: v = gs[(size_t)tau * N + u]; break;
            case 1: v = gs[(size_t)tau * N + (N - 1 - u)]; break;
            case 2: v = gs[(size_t)u * N + tau]; break;
            default: v = gs[(size_t)(N - 1 - u) * N + tau]; break;
        }
    }
    A[((size_t)sq * N + tau) * W + u] = v;
}

// One transposed stage: level k (strips of 2^k rows) -> level k-1.  Rows are stored strip
// after strip, row b 2^k + tau of level k holding A_k[b][tau].
__global__ void __launch_bounds__(kAdjThreads)
adj_stage_kernel(const float* __restrict__ in, float* __restrict__ out, int N, int W, int k)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;                   // output row at level k-1
    const size_t base = (size_t)blockIdx.z * N * W;
    if (v >= W) return;
    const int h = 1 << (k - 1);
    const int bc = r >> (k - 1);                // child strip at level k-1
    const int t = r & (h - 1);
    const int r0 = ((bc >> 1) << k) + 2 * t;    // A_k[bc / 2][2t]; r0 + 1 is A_k[bc / 2][2t + 1]
    const float* a0 = in + base + (size_t)r0 * W;
    const float* a1 = a0 + W;
    float o;
    if ((bc & 1) == 0) {
        o = a0[v] + a1[v];
    } else {
        const float x0 = v >= t ? a0[v - t] : 0.0f;
        const float x1 = v >= t + 1 ? a1[v - t - 1] : 0.0f;
        o = x0 + x1;
    }
    out[base + (size_t)r * W + v] = o;
}

// Transposed resampling: every linogram sample's gradient into the four sinogram bins of
// its bilinear interpolation (same fixed-point positions and float32 weights as the forward
// resampling).  Samples of value zero (all of them outside the trapezoid) add nothing.
__global__ void __launch_bounds__(kAdjThreads)
adj_resample_kernel(const float* __restrict__ lbar, float* __restrict__ pbar,
                    const RowGeom* __restrict__ geom, int N, int K, int M)
{
    const int W = 2 * N;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int qi = blockIdx.y;                  // q * N + i
    const int s = blockIdx.z;
    if (c >= W) return;
    const float val = lbar[((size_t)s * 4 * N + qi) * W + c];
    if (val == 0.0f) return;
    const RowGeom gm = geom[qi];
    float* ps = pbar + (size_t)s * K * M;
    const long long m = gm.b_fx + gm.a_fx * (long long)c;
    const int j = (int)(m >> kFixBits);
    const float f = __uint2float_rn((unsigned)m) * 0x1p-32f;
    float* ra = ps + (size_t)gm.k0 * M;
    const float va = gm.w0 * val;               // gradient of the k0 lerp
    if (j >= 0 && j < M) atomicAdd(ra + j, va * (1.0f - f));
    if (j + 1 >= 0 && j + 1 < M) atomicAdd(ra + j + 1, va * f);
    const float vb = gm.w1 * val;
    if (!gm.wrap) {
        float* rb = ra + M;
        if (j >= 0 && j < M) atomicAdd(rb + j, vb * (1.0f - f));
        if (j + 1 >= 0 && j + 1 < M) atomicAdd(rb + j + 1, vb * f);
    } else {                                    // row 0, detector mirrored: m' = M-1-m
        const long long mm = ((long long)(M - 1) << kFixBits) - m;
        const int jm = (int)(mm >> kFixBits);
        const float fm = __uint2float_rn((unsigned)mm) * 0x1p-32f;
        if (jm >= 0 && jm < M) atomicAdd(ps + jm, vb * (1.0f - fm));
        if (jm + 1 >= 0 && jm + 1 < M) atomicAdd(ps + jm + 1, vb * fm);
    }
}

}  // namespace

cudaError_t launch_fht_adjoint(const fbp_plan_s* p, const float* img_grad, float* lin_grad,
                               float* scratch, int count, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    const int N = p->N, W = 2 * N, n = p->n;
    // n stages after the quarter step: start in the buffer that makes the last stage land
    // in lin_grad
    float* buf[2] = {lin_grad, scratch};
    int cur = (n & 1) ? 1 : 0;
    const dim3 blk(kAdjThreads);
    adj_quarters_kernel<<<dim3((W + kAdjThreads - 1) / kAdjThreads, N, 4 * count), blk, 0, st>>>(
        img_grad, buf[cur], N, W);
    cudaError_t e = cudaGetLastError();
    for (int k = n; k >= 1 && e == cudaSuccess; --k) {
        adj_stage_kernel<<<dim3((W + kAdjThreads - 1) / kAdjThreads, N, 4 * count), blk, 0, st>>>(
            buf[cur], buf[cur ^ 1], N, W, k);
        cur ^= 1;
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_resample_adjoint(const fbp_plan_s* p, const float* lin_grad, float* filt_grad,
                                    int count, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(filt_grad, 0, (size_t)count * p->K * p->M * sizeof(float), st);
    if (e != cudaSuccess) return e;
    adj_resample_kernel<<<dim3((2 * p->N + kAdjThreads - 1) / kAdjThreads, 4 * p->N, count),
                          kAdjThreads, 0, st>>>(lin_grad, filt_grad, p->d_geom, p->N, p->K, p->M);
    return cudaGetLastError();
}

}  // namespace fbp
