// Direct FBP, the comparator of the fast method (paper Sec. 2, Eq. 3-5 and Eq. 8):
//   p~(n) = sum_{k=-(M-1)}^{M-1} h(k) p(n-k),  h of Eq. 7 (exact convolution of the row)
//   f(x, y) = (pi/K) sum_k lerp(p~_k, (x-c0) cos(theta_k) + (y-c0) sin(theta_k) + (M-1)/2)
// Theta(K M^2) for the filter and Theta(K N^2) for the back projection.
#include "fbp_internal.h"

namespace fbp {
namespace {

constexpr float kInvPi2 = 0.10132118364233778f;    // 1 / pi^2

// One CTA per row: the row and the kernel taps h(|d|) live in shared memory.  h(d) is
// zero for even d != 0, so each output sums over the detector bins of opposite parity.
__global__ void __launch_bounds__(256)
fir_ramp_kernel(const float* __restrict__ in, float* __restrict__ out, int M)
{
    extern __shared__ float sm[];
    float* sp = sm;
    float* sh = sm + M;
    const size_t row = blockIdx.x;
    const float* src = in + row * M;
    for (int n = threadIdx.x; n < M; n += blockDim.x) {
        sp[n] = src[n];
        const float d = (float)n;
        sh[n] = (n == 0) ? 0.25f : ((n & 1) ? -kInvPi2 / (d * d) : 0.0f);
    }
    __syncthreads();
    for (int n = threadIdx.x; n < M; n += blockDim.x) {
        float acc = 0.25f * sp[n];
        for (int j = (n & 1) ? 0 : 1; j < M; j += 2) {
            const int d = n > j ? n - j : j - n;
            acc = fmaf(sp[j], sh[d], acc);
        }
        out[row * M + n] = acc;
    }
}

constexpr int kBpTile = 16;
constexpr int kBpTrig = 256;

// Pixel-driven back projection: one thread per pixel, angles streamed through a shared
// table of (cos, sin).
__global__ void __launch_bounds__(kBpTile * kBpTile)
direct_bp_kernel(const float* __restrict__ filt, float* __restrict__ img,
                 const float2* __restrict__ trig, int N, int K, int M)
{
    __shared__ float2 st[kBpTrig];
    const int x = blockIdx.x * kBpTile + threadIdx.x;
    const int y = blockIdx.y * kBpTile + threadIdx.y;
    const int s = blockIdx.z;
    const int tid = threadIdx.y * kBpTile + threadIdx.x;
    const float c0 = 0.5f * (float)(N - 1);
    const float xc = (float)x - c0;
    const float yc = (float)y - c0;
    const float half = 0.5f * (float)(M - 1);
    const float* pt = filt + (size_t)s * K * M;
    float acc = 0.0f;
    for (int k0 = 0; k0 < K; k0 += kBpTrig) {
        __syncthreads();
        if (k0 + tid < K && tid < kBpTrig) st[tid] = trig[k0 + tid];
        __syncthreads();
        const int kn = min(kBpTrig, K - k0);
        for (int kk = 0; kk < kn; ++kk) {
            const float2 cs = st[kk];
            const float m = fmaf(xc, cs.x, fmaf(yc, cs.y, half));
            const float fl = floorf(m);
            const int j = (int)fl;
            const float f = m - fl;
            const float* row = pt + (size_t)(k0 + kk) * M;
            const float v0 = (j >= 0 && j < M) ? __ldg(row + j) : 0.0f;
            const float v1 = (j + 1 >= 0 && j + 1 < M) ? __ldg(row + j + 1) : 0.0f;
            acc += fmaf(f, v1 - v0, v0);
        }
    }
    if (x < N && y < N) img[((size_t)s * N + y) * N + x] = acc * (3.14159265358979323846f / (float)K);
}

}  // namespace

cudaError_t prepare_direct_kernels()
{
    return cudaFuncSetAttribute(fir_ramp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                227 * 1024);
}

cudaError_t launch_fir(const fbp_plan_s* p, const float* in, float* out, int rows,
                       cudaStream_t st)
{
    if (rows <= 0) return cudaSuccess;
    const size_t smem = (size_t)2 * p->M * sizeof(float);
    fir_ramp_kernel<<<rows, 256, smem, st>>>(in, out, p->M);
    return cudaGetLastError();
}

cudaError_t launch_direct_bp(const fbp_plan_s* p, const float* filt, float* img, int count,
                             cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    dim3 block(kBpTile, kBpTile);
    dim3 grid((p->N + kBpTile - 1) / kBpTile, (p->N + kBpTile - 1) / kBpTile, count);
    direct_bp_kernel<<<grid, block, 0, st>>>(filt, img, p->d_trig, p->N, p->K, p->M);
    return cudaGetLastError();
}

}  // namespace fbp
