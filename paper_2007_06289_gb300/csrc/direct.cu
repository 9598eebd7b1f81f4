// Direct FBP, the comparator of the fast method (paper Sec. 2, Eq. 3-5 and Eq. 8):
//   p~(n) = sum_{k=-(M-1)}^{M-1} h(k) p(n-k),  h of Eq. 7 (exact convolution of the row)
//   f(x, y) = (pi/K) sum_k lerp(p~_k, (x-c0) cos(theta_k) + (y-c0) sin(theta_k) + (M-1)/2)
// Theta(K M^2) for the filter and Theta(K N^2) for the back projection.
#include "fbp_internal.h"

namespace fbp {
namespace {

constexpr float kInvPi2 = 0.10132118364233778f;    // 1 / pi^2

// Exact ramp filter, one CTA per row.  p~(n) = p(n)/4 + sum_{e odd, |e| <= M-1} h(e) p(n - e),
// h(e) = -1/(pi e)^2 (h vanishes at even e != 0).  The row sits in shared memory with zeros on
// both sides (so p(n - e) needs no range test) and the odd taps in ascending e.  Each thread
// computes 4 consecutive outputs n0 .. n0 + 3 and walks the taps 4 at a time: the samples
// p(n0 - e - 4 .. n0 - e + 3) it needs form a window that moves down by 4 per 2 taps, so each
// 2 taps cost one 16-byte load of 4 new samples (the row is stored shifted so that these
// loads are aligned) and 8 FMAs, and 4 taps one 16-byte broadcast of h.  Θ(M^2) per row.
constexpr int kFirThreads = 256;
constexpr int kFirG = 4;                          // outputs per thread

__host__ __device__ inline int fir_first_tap(int M)
{
    // the first tap offset: odd, congruent to 3 mod 4, at most -(M - 1)
    int e = -(M - 1) - 4;
    while (((e % 4) + 4) % 4 != 3) ++e;
    return e;
}

__host__ __device__ inline int fir_taps(int M)     // taps per row, a multiple of 4
{
    const int e0 = fir_first_tap(M);
    const int n = ((M - 1) - e0) / 2 + 1;
    return (n + 3) & ~3;
}

// shared floats: the taps, then the row with (M + 16) zeros before and after
__host__ __device__ inline int fir_off(int M) { return ((M + 16) & ~3) + 3; }   // = 3 mod 4
__host__ __device__ inline size_t fir_smem_floats(int M)
{
    return (size_t)fir_taps(M) + (size_t)fir_off(M) + (size_t)M + (size_t)M + 24;
}

__global__ void __launch_bounds__(kFirThreads)
fir_ramp_kernel(const float* __restrict__ in, float* __restrict__ out, int M)
{
    extern __shared__ __align__(16) float sm[];
    const int T = fir_taps(M);
    const int e0 = fir_first_tap(M);
    const int off = fir_off(M);
    float* hs = sm;                                   // hs[i] = h(e0 + 2 i)
    float* ps = sm + T;                               // ps[off + k] = p(k)
    const int len = off + M + M + 24;
    const size_t row = blockIdx.x;
    const float* src = in + row * M;
    for (int i = threadIdx.x; i < T; i += blockDim.x) {
        const int e = e0 + 2 * i;
        const float d = (float)e;
        hs[i] = (e >= -(M - 1) && e <= M - 1) ? -kInvPi2 / (d * d) : 0.0f;
    }
    for (int k = threadIdx.x; k < len; k += blockDim.x) {
        const int n = k - off;
        ps[k] = (n >= 0 && n < M) ? src[n] : 0.0f;
    }
    __syncthreads();
    for (int n0 = kFirG * threadIdx.x; n0 < M; n0 += kFirG * blockDim.x) {
        float acc[kFirG] = {0.0f, 0.0f, 0.0f, 0.0f};
        // window w[0..7] = p(n0 - e - 4 .. n0 - e + 3) for the current tap e
        const float* base = ps + off + n0;
        float4 lo = *reinterpret_cast<const float4*>(base - e0 - 4);
        float4 hi = *reinterpret_cast<const float4*>(base - e0);
        for (int i = 0; i < T; i += 4) {
            const int e = e0 + 2 * i;
            const float4 h = *reinterpret_cast<const float4*>(hs + i);   // h(e), h(e+2), h(e+4), h(e+6)
            const float w[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
            // tap e: p(n0 + g - e) = w[4 + g]; tap e + 2: p(n0 + g - e - 2) = w[2 + g]
#pragma unroll
            for (int g = 0; g < kFirG; ++g) acc[g] = fmaf(h.x, w[4 + g], acc[g]);
#pragma unroll
            for (int g = 0; g < kFirG; ++g) acc[g] = fmaf(h.y, w[2 + g], acc[g]);
            const float4 u = *reinterpret_cast<const float4*>(base - e - 8);   // p(n0 - e - 8 ..)
            // taps e + 4 and e + 6 on the window p(n0 - e - 8 .. n0 - e - 1) = (u, lo)
            const float v[8] = {u.x, u.y, u.z, u.w, lo.x, lo.y, lo.z, lo.w};
#pragma unroll
            for (int g = 0; g < kFirG; ++g) acc[g] = fmaf(h.z, v[4 + g], acc[g]);
#pragma unroll
            for (int g = 0; g < kFirG; ++g) acc[g] = fmaf(h.w, v[2 + g], acc[g]);
            hi = lo;
            lo = *reinterpret_cast<const float4*>(base - e - 12);            // p(n0 - e - 12 ..)
            hi = u;
        }
#pragma unroll
        for (int g = 0; g < kFirG; ++g)
            if (n0 + g < M) out[row * M + n0 + g] = fmaf(0.25f, ps[off + n0 + g], acc[g]);
    }
}

// The same filter for rows too long for the blocked form's padded row (M above ~14,000): one
// output per thread, taps and samples read from shared memory term by term.
__global__ void __launch_bounds__(256)
fir_ramp_long_kernel(const float* __restrict__ in, float* __restrict__ out, int M)
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

// Pixel-driven back projection.  CTA = 32 x 32 pixels, 256 threads, each thread 4 pixels of
// one column (rows ty, ty + 8, ty + 16, ty + 24).  Angles go in blocks of kBpA: for each
// angle of a block the detector window the tile reads (at most 31 (|cos| + |sin|) + 2 <= 46
// bins wide, staged as kBpW bins from one below the lowest position) is copied into shared
// memory with zeros outside [0, M), so the inner loop reads shared memory only.  Every
// pixel's sum runs over the angles in order with the arithmetic of the plain per-pixel form.
constexpr int kBpT = 32;
constexpr int kBpRows = 4;                       // pixels per thread
constexpr int kBpThreads = kBpT * kBpT / kBpRows;
constexpr int kBpA = 32;                         // angles per staged block
constexpr int kBpW = 64;                         // staged bins per angle

__global__ void __launch_bounds__(kBpThreads)
direct_bp_kernel(const float* __restrict__ filt, float* __restrict__ img,
                 const float2* __restrict__ trig, int N, int K, int M)
{
    __shared__ float win[kBpA][kBpW];
    __shared__ float2 scs[kBpA];
    __shared__ int sjb[kBpA];
    const int tid = threadIdx.x;
    const int tx = tid % kBpT, ty = tid / kBpT;
    const int xb = blockIdx.x * kBpT, yb = blockIdx.y * kBpT;
    const int s = blockIdx.z;
    const float c0 = 0.5f * (float)(N - 1);
    const float half = 0.5f * (float)(M - 1);
    const float xc = (float)(xb + tx) - c0;
    float yc[kBpRows], acc[kBpRows];
#pragma unroll
    for (int r = 0; r < kBpRows; ++r) {
        yc[r] = (float)(yb + ty + (kBpT / kBpRows) * r) - c0;
        acc[r] = 0.0f;
    }
    const float* pt = filt + (size_t)s * K * M;
    for (int k0 = 0; k0 < K; k0 += kBpA) {
        const int ka = min(kBpA, K - k0);
        __syncthreads();                                 // previous block consumed
        if (tid < ka) {
            const float2 cs = trig[k0 + tid];
            // lowest detector position over the tile's corners, one bin of slack below
            const float xl = (float)xb - c0, xh = xl + (float)(kBpT - 1);
            const float yl = (float)yb - c0, yh = yl + (float)(kBpT - 1);
            const float mlo = fminf(fminf(fmaf(xl, cs.x, fmaf(yl, cs.y, half)), fmaf(xh, cs.x, fmaf(yl, cs.y, half))),
                                    fminf(fmaf(xl, cs.x, fmaf(yh, cs.y, half)), fmaf(xh, cs.x, fmaf(yh, cs.y, half))));
            scs[tid] = cs;
            sjb[tid] = (int)floorf(mlo) - 1;
        }
        __syncthreads();
        for (int e = tid; e < ka * kBpW; e += kBpThreads) {
            const int a = e / kBpW, b = e - a * kBpW;
            const int j = sjb[a] + b;
            win[a][b] = (j >= 0 && j < M) ? __ldg(pt + (size_t)(k0 + a) * M + j) : 0.0f;
        }
        __syncthreads();
        for (int a = 0; a < ka; ++a) {
            const float2 cs = scs[a];
            const int jb = sjb[a];
            const float* wr = win[a];
#pragma unroll
            for (int r = 0; r < kBpRows; ++r) {
                const float m = fmaf(xc, cs.x, fmaf(yc[r], cs.y, half));
                const float fl = floorf(m);
                const int jl = min(max((int)fl - jb, 0), kBpW - 2);
                const float f = m - fl;
                const float v0 = wr[jl], v1 = wr[jl + 1];
                acc[r] += fmaf(f, v1 - v0, v0);
            }
        }
    }
    const int x = xb + tx;
#pragma unroll
    for (int r = 0; r < kBpRows; ++r) {
        const int y = yb + ty + (kBpT / kBpRows) * r;
        if (x < N && y < N) img[((size_t)s * N + y) * N + x] = acc[r] * (3.14159265358979323846f / (float)K);
    }
}

}  // namespace

cudaError_t prepare_direct_kernels()
{
    cudaError_t e = cudaFuncSetAttribute(fir_ramp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         227 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fir_ramp_long_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 227 * 1024);
    return e;
}

cudaError_t launch_fir(const fbp_plan_s* p, const float* in, float* out, int rows,
                       cudaStream_t st)
{
    if (rows <= 0) return cudaSuccess;
    const size_t smem = fir_smem_floats(p->M) * sizeof(float);
    if (smem <= (size_t)227 * 1024) {
        fir_ramp_kernel<<<rows, kFirThreads, smem, st>>>(in, out, p->M);
    } else {
        const size_t smem2 = (size_t)2 * p->M * sizeof(float);
        fir_ramp_long_kernel<<<rows, 256, smem2, st>>>(in, out, p->M);
    }
    return cudaGetLastError();
}

cudaError_t launch_direct_bp(const fbp_plan_s* p, const float* filt, float* img, int count,
                             cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    dim3 grid((p->N + kBpT - 1) / kBpT, (p->N + kBpT - 1) / kBpT, count);
    direct_bp_kernel<<<grid, kBpThreads, 0, st>>>(filt, img, p->d_trig, p->N, p->K, p->M);
    return cudaGetLastError();
}

}  // namespace fbp
