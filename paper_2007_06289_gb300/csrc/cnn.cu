// Learned residual corrector after the fast reconstruction: six 3x3 convolutions
// (1 -> 32 -> 32 -> 32 -> 32 -> 32 -> 1 channels, ReLU between, zero padding) whose output
// is added to the input image, y = x + net(x); forward and gradients for training.
//
// Data layout: hidden activations are bf16 [batch][N][N][32], channel fastest (one pixel's
// 32 channels are 64 contiguous bytes).  The four 32 -> 32 layers run on the tensor cores
// as implicit GEMMs (pixels x output channels x (taps x input channels), bf16 operands,
// fp32 accumulation, mma.sync m16n8k16 fed by ldmatrix from padded shared tiles, persistent
// CTAs with double-buffered asynchronous tile loads); the
// 1 -> 32 and 32 -> 1 layers, the last layer's gradient and the weight gradients run on the
// CUDA cores in fp32.  The data gradient of a 32 -> 32 layer is the same tensor-core kernel
// with the layer's weights transposed (input and output channels swapped, taps mirrored)
// and the previous layer's ReLU applied as a mask.
//
// Parameters: one fp32 array, layer after layer, each layer's weights [co][ci][3][3]
// followed by its biases [co].
#include <cuda_bf16.h>

#include <mutex>

#include "fbp_internal.h"

namespace fbp {
namespace {

constexpr int kC = 32;            // hidden channels
constexpr int kTaps = 9;
constexpr int kK = kC * kTaps;    // GEMM depth of a 32 -> 32 layer
constexpr int kTileY = 8, kTileX = 16;           // pixels per tile of the weight-gradient kernel
constexpr int kHaloY = kTileY + 2, kHaloX = kTileX + 2;
constexpr int kPixStride = 40;    // bf16 per shared pixel (80 bytes: conflict-free ldmatrix)
constexpr int kWStride = kK + 8;  // bf16 per shared weight row (592 bytes: conflict-free)

using bf16 = __nv_bfloat16;

__device__ __forceinline__ unsigned smem_u32(const void* p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldmatrix_x4(unsigned (&r)[4], const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0,
                                         unsigned b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                 "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// ---------------------------------------------------------------- weight preparation
// fp32 [co][ci][3][3] of a 32 -> 32 layer -> bf16 GEMM rows: forward [co][tap][ci]; for the
// data gradient [ci][8 - tap][co] (the transposed convolution).
__global__ void cnn_prep_weights_kernel(const float* __restrict__ w, bf16* __restrict__ fwd,
                                        bf16* __restrict__ bwd)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;      // co, ci, tap
    if (e >= kC * kC * kTaps) return;
    const int tap = e % kTaps;
    const int ci = (e / kTaps) % kC;
    const int co = e / (kTaps * kC);
    const bf16 v = __float2bfloat16_rn(w[e]);
    fwd[(size_t)co * kK + tap * kC + ci] = v;
    bwd[(size_t)ci * kK + (kTaps - 1 - tap) * kC + co] = v;
}

// ---------------------------------------------------------------- 32 -> 32 on tensor cores
// out[p][o] = bias[o] + sum_{tap, c} W[o][tap][c] in[p + off(tap)][c], optional ReLU, optional
// mask (out *= mask[p][o] > 0).  Persistent CTAs: the layer's weights are staged once per
// CTA; the CTA then walks 16 x 16-pixel output tiles, the next tile's input (with its
// one-pixel halo) arriving by asynchronous copies into the second of two shared buffers
// while the tensor cores work on the current one.  Warp w computes output rows 2w and 2w+1
// of a tile (two 16-pixel M tiles sharing every weight fragment).
constexpr int kT2 = 16;                           // output tile: 16 x 16 pixels
constexpr int kH2 = kT2 + 2;                      // with the halo
constexpr int kActElems = kH2 * kH2 * kPixStride; // bf16 per activation buffer
constexpr size_t kConvSmem = (size_t)(kC * kWStride + 2 * kActElems) * sizeof(bf16);

__device__ __forceinline__ void cp_async16z(void* dst, const void* src, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)),
                 "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}

// the input tile of output tile t (image, ty, tx) with its halo, zero outside the image
__device__ __forceinline__ void conv_prefetch(bf16* act, const bf16* in, long long t, int N,
                                              int tiles_x, int tiles_per_img, int tid)
{
    const int im = (int)(t / tiles_per_img);
    const int rem = (int)(t - (long long)im * tiles_per_img);
    const int y0 = (rem / tiles_x) * kT2, x0 = (rem % tiles_x) * kT2;
    const size_t img = (size_t)im * N * N;
    for (int e = tid; e < kH2 * kH2 * 4; e += 256) {
        const int pix = e >> 2, part = e & 3;
        const int ty = pix / kH2, tx = pix - ty * kH2;
        const int gy = y0 - 1 + ty, gx = x0 - 1 + tx;
        const bool ok = gy >= 0 && gy < N && gx >= 0 && gx < N;
        const bf16* src = ok ? in + (img + (size_t)gy * N + gx) * kC + part * 8 : in;
        cp_async16z(act + pix * kPixStride + part * 8, src, ok);
    }
}

template <bool BIAS, bool RELU, bool MASK>
__global__ void __launch_bounds__(256)
cnn_conv32_kernel(const bf16* __restrict__ in, const bf16* __restrict__ wt,
                  const float* __restrict__ bias, const bf16* __restrict__ mask,
                  bf16* __restrict__ out, int N, int images)
{
    extern __shared__ __align__(16) unsigned char conv_smem[];
    bf16* wsm = reinterpret_cast<bf16*>(conv_smem);
    bf16* act0 = wsm + kC * kWStride;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_x = N / kT2, tiles_per_img = tiles_x * (N / kT2);
    const long long total = (long long)tiles_per_img * images;

    for (int e = tid; e < kC * (kK / 8); e += 256) {
        const int row = e / (kK / 8), part = e - row * (kK / 8);
        *reinterpret_cast<uint4*>(wsm + row * kWStride + part * 8) =
            *reinterpret_cast<const uint4*>(wt + (size_t)row * kK + part * 8);
    }
    long long t = blockIdx.x;
    if (t < total) conv_prefetch(act0, in, t, N, tiles_x, tiles_per_img, tid);
    asm volatile("cp.async.commit_group;\n" ::: "memory");

    const int j = lane >> 3, r = lane & 7;
    const int g = lane >> 2, q4 = lane & 3;
    for (int it = 0; t < total; ++it, t += gridDim.x) {
        bf16* act = act0 + (it & 1) * kActElems;
        const long long tn = t + gridDim.x;
        if (tn < total)
            conv_prefetch(act0 + ((it + 1) & 1) * kActElems, in, tn, N, tiles_x, tiles_per_img, tid);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        __syncthreads();

        float acc[2][4][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[mt][nt][k] = 0.0f;
#pragma unroll 1
        for (int tap = 0; tap < kTaps; ++tap) {
            const int dy = tap / 3, dx = tap - 3 * (tap / 3);
#pragma unroll
            for (int cb = 0; cb < 2; ++cb) {
                unsigned a[2][4];
                const int xx = r + 8 * (j & 1);
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
                    ldmatrix_x4(a[mt], act + ((2 * warp + mt + dy) * kH2 + xx + dx) * kPixStride +
                                           cb * 16 + 8 * (j >> 1));
                const int kb = tap * kC + cb * 16;
#pragma unroll
                for (int pr = 0; pr < 2; ++pr) {
                    unsigned bb[4];
                    ldmatrix_x4(bb, wsm + ((2 * pr + (j >> 1)) * 8 + r) * kWStride + kb + 8 * (j & 1));
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt) {
                        mma_bf16(acc[mt][2 * pr], a[mt], bb[0], bb[1]);
                        mma_bf16(acc[mt][2 * pr + 1], a[mt], bb[2], bb[3]);
                    }
                }
            }
        }

        const int im = (int)(t / tiles_per_img);
        const int rem = (int)(t - (long long)im * tiles_per_img);
        const int y0 = (rem / tiles_x) * kT2, x0 = (rem % tiles_x) * kT2;
        const size_t img = (size_t)im * N * N;
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const int py = y0 + 2 * warp + mt;
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int ch = nt * 8 + 2 * q4;
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    const int px = x0 + g + 8 * half;
                    const size_t p = (img + (size_t)py * N + px) * kC + ch;
                    float v0 = acc[mt][nt][2 * half], v1 = acc[mt][nt][2 * half + 1];
                    if (BIAS) { v0 += bias[ch]; v1 += bias[ch + 1]; }
                    if (RELU) { v0 = fmaxf(v0, 0.0f); v1 = fmaxf(v1, 0.0f); }
                    if (MASK) {
                        const float2 m = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(mask + p));
                        v0 = m.x > 0.0f ? v0 : 0.0f;
                        v1 = m.y > 0.0f ? v1 : 0.0f;
                    }
                    *reinterpret_cast<__nv_bfloat162*>(out + p) = __floats2bfloat162_rn(v0, v1);
                }
            }
        }
        __syncthreads();                          // this buffer is refilled two tiles on
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// ---------------------------------------------------------------- 1 -> 32 and 32 -> 1
// First layer: h[p][o] = relu(b[o] + sum_tap w[o][tap] x[p + off(tap)]), fp32 math.
__global__ void __launch_bounds__(256)
cnn_first_kernel(const float* __restrict__ x, const float* __restrict__ w,
                 const float* __restrict__ b, bf16* __restrict__ h, int N)
{
    __shared__ float ws[kC * kTaps + kC];
    for (int e = threadIdx.x; e < kC * kTaps + kC; e += blockDim.x) ws[e] = w[e];  // w then b
    __syncthreads();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N * N) return;
    const int py = p / N, px = p - py * N;
    const float* xs = x + (size_t)blockIdx.y * N * N;
    float v[kTaps];
#pragma unroll
    for (int tap = 0; tap < kTaps; ++tap) {
        const int yy = py + tap / 3 - 1, xx = px + tap % 3 - 1;
        v[tap] = (yy >= 0 && yy < N && xx >= 0 && xx < N) ? xs[(size_t)yy * N + xx] : 0.0f;
    }
    (void)b;
    uint4 pk[4];
    unsigned* pw = reinterpret_cast<unsigned*>(pk);
#pragma unroll
    for (int o = 0; o < kC; o += 2) {
        float s0 = ws[kC * kTaps + o], s1 = ws[kC * kTaps + o + 1];
#pragma unroll
        for (int tap = 0; tap < kTaps; ++tap) {
            s0 = fmaf(ws[o * kTaps + tap], v[tap], s0);
            s1 = fmaf(ws[(o + 1) * kTaps + tap], v[tap], s1);
        }
        const __nv_bfloat162 q = __floats2bfloat162_rn(fmaxf(s0, 0.0f), fmaxf(s1, 0.0f));
        pw[o >> 1] = *reinterpret_cast<const unsigned*>(&q);
    }
    uint4* dst = reinterpret_cast<uint4*>(h + ((size_t)blockIdx.y * N * N + p) * kC);
#pragma unroll
    for (int k = 0; k < 4; ++k) dst[k] = pk[k];
}

__device__ __forceinline__ void load_pixel32(float (&v)[kC], const bf16* src)
{
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint4 q = s4[k];
        const unsigned u[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u[m]));
            v[8 * k + 2 * m] = f.x;
            v[8 * k + 2 * m + 1] = f.y;
        }
    }
}

// Last layer and the skip connection: y[p] = x[p] + b + sum_{tap, c} w[c][tap] h[p + off][c].
__global__ void __launch_bounds__(256)
cnn_last_kernel(const float* __restrict__ x, const bf16* __restrict__ h, const float* __restrict__ w,
                float* __restrict__ y, int N)
{
    __shared__ float ws[kC * kTaps + 1];
    for (int e = threadIdx.x; e < kC * kTaps + 1; e += blockDim.x) ws[e] = w[e];   // w then b
    __syncthreads();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N * N) return;
    const int py = p / N, px = p - py * N;
    const size_t img = (size_t)blockIdx.y * N * N;
    float s = ws[kC * kTaps];
    for (int tap = 0; tap < kTaps; ++tap) {
        const int yy = py + tap / 3 - 1, xx = px + tap % 3 - 1;
        if (yy < 0 || yy >= N || xx < 0 || xx >= N) continue;
        float v[kC];
        load_pixel32(v, h + (img + (size_t)yy * N + xx) * kC);
#pragma unroll
        for (int c = 0; c < kC; ++c) s = fmaf(ws[c * kTaps + tap], v[c], s);
    }
    y[img + p] = x[img + p] + s;
}

// Gradient through the last layer into the fifth layer's pre-activation:
// g[p][c] = (h5[p][c] > 0) * sum_tap w[c][tap] gy[p - off(tap)].
__global__ void __launch_bounds__(256)
cnn_last_backward_kernel(const float* __restrict__ gy, const bf16* __restrict__ h5,
                         const float* __restrict__ w, bf16* __restrict__ g, int N)
{
    __shared__ float ws[kC * kTaps];
    for (int e = threadIdx.x; e < kC * kTaps; e += blockDim.x) ws[e] = w[e];
    __syncthreads();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N * N) return;
    const int py = p / N, px = p - py * N;
    const size_t img = (size_t)blockIdx.y * N * N;
    float v[kTaps];
#pragma unroll
    for (int tap = 0; tap < kTaps; ++tap) {
        const int yy = py - (tap / 3 - 1), xx = px - (tap % 3 - 1);
        v[tap] = (yy >= 0 && yy < N && xx >= 0 && xx < N) ? gy[img + (size_t)yy * N + xx] : 0.0f;
    }
    float m[kC];
    load_pixel32(m, h5 + (img + p) * kC);
    uint4 pk[4];
    unsigned* pw = reinterpret_cast<unsigned*>(pk);
#pragma unroll
    for (int c = 0; c < kC; c += 2) {
        float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
        for (int tap = 0; tap < kTaps; ++tap) {
            s0 = fmaf(ws[c * kTaps + tap], v[tap], s0);
            s1 = fmaf(ws[(c + 1) * kTaps + tap], v[tap], s1);
        }
        const __nv_bfloat162 q = __floats2bfloat162_rn(m[c] > 0.0f ? s0 : 0.0f,
                                                       m[c + 1] > 0.0f ? s1 : 0.0f);
        pw[c >> 1] = *reinterpret_cast<const unsigned*>(&q);
    }
    uint4* dst = reinterpret_cast<uint4*>(g + (img + p) * kC);
#pragma unroll
    for (int k = 0; k < 4; ++k) dst[k] = pk[k];
}

// ---------------------------------------------------------------- weight gradients (fp32)
// gw[o][c][tap] += sum_p gz[p][o] hp[p + off(tap)][c], gb[o] += sum_p gz[p][o], over all pixels
// of all images.  CO / CI are 32 or 1; a 1-channel operand is fp32 [N][N] (the image or the
// output gradient), a 32-channel one bf16 [N][N][32].  Persistent CTAs accumulate over
// 8 x 16-pixel tiles in registers and add once into the global gradient.
template <int CO, int CI>
__global__ void __launch_bounds__(256)
cnn_wgrad_kernel(const void* __restrict__ gz_, const void* __restrict__ hp_, float* __restrict__ gw,
                 float* __restrict__ gb, int N, int images)
{
    constexpr int NOUT = CO * CI * kTaps;
    constexpr int PER = (NOUT + 255) / 256;
    __shared__ float gzs[kTileY * kTileX][CO];
    __shared__ float hps[kHaloY * kHaloX][CI];
    const int tid = threadIdx.x;
    float acc[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) acc[k] = 0.0f;
    float accb = 0.0f;
    const int tiles_x = N / kTileX, tiles_y = N / kTileY;
    const long long tiles = (long long)tiles_x * tiles_y * images;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int im = (int)(tile / ((long long)tiles_x * tiles_y));
        const int rem = (int)(tile - (long long)im * tiles_x * tiles_y);
        const int y0 = (rem / tiles_x) * kTileY, x0 = (rem % tiles_x) * kTileX;
        const size_t img = (size_t)im * N * N;
        __syncthreads();                               // previous tile consumed
        for (int e = tid; e < kTileY * kTileX * CO; e += 256) {
            const int pix = e / CO, o = e - pix * CO;
            const size_t gp = img + (size_t)(y0 + pix / kTileX) * N + x0 + pix % kTileX;
            gzs[pix][o] = CO == 1 ? static_cast<const float*>(gz_)[gp]
                                  : __bfloat162float(static_cast<const bf16*>(gz_)[gp * kC + o]);
        }
        for (int e = tid; e < kHaloY * kHaloX * CI; e += 256) {
            const int pix = e / CI, c = e - pix * CI;
            const int gy = y0 - 1 + pix / kHaloX, gx = x0 - 1 + pix % kHaloX;
            float v = 0.0f;
            if (gy >= 0 && gy < N && gx >= 0 && gx < N) {
                const size_t gp = img + (size_t)gy * N + gx;
                v = CI == 1 ? static_cast<const float*>(hp_)[gp]
                            : __bfloat162float(static_cast<const bf16*>(hp_)[gp * kC + c]);
            }
            hps[pix][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int e = tid + 256 * k;               // (o, c, tap) in parameter order
            if (e < NOUT) {
                const int tap = e % kTaps, c = (e / kTaps) % CI, o = e / (kTaps * CI);
                const int dy = tap / 3, dx = tap % 3;
                float s = acc[k];
                for (int pix = 0; pix < kTileY * kTileX; ++pix) {
                    const int py = pix / kTileX, px = pix % kTileX;
                    s = fmaf(gzs[pix][o], hps[(py + dy) * kHaloX + px + dx][c], s);
                }
                acc[k] = s;
            }
        }
        if (tid < CO)
            for (int pix = 0; pix < kTileY * kTileX; ++pix) accb += gzs[pix][tid];
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int e = tid + 256 * k;
        if (e < NOUT) atomicAdd(gw + e, acc[k]);
    }
    if (tid < CO) atomicAdd(gb + tid, accb);
}

}  // namespace

// ---------------------------------------------------------------- host side
namespace cnn {

constexpr int kLayers = 6;

size_t param_count()
{
    size_t n = 0;
    for (int k = 0; k < kLayers; ++k) {
        const int ci = k == 0 ? 1 : kC, co = k == kLayers - 1 ? 1 : kC;
        n += (size_t)co * ci * kTaps + co;
    }
    return n;
}

size_t param_offset(int layer)
{
    size_t n = 0;
    for (int k = 0; k < layer; ++k) {
        const int ci = k == 0 ? 1 : kC, co = k == kLayers - 1 ? 1 : kC;
        n += (size_t)co * ci * kTaps + co;
    }
    return n;
}

size_t act_bytes(int N, int batch) { return (size_t)batch * N * N * kC * sizeof(bf16); }

// workspace: bf16 GEMM weights (4 layers x forward and transposed), then `nact` activation
// buffers and 2 gradient buffers
size_t workspace_bytes(int N, int batch, int train)
{
    const size_t wbytes = (size_t)4 * 2 * kC * kK * sizeof(bf16);
    const int nbuf = train ? 5 + 2 : 2;
    return wbytes + (size_t)nbuf * act_bytes(N, batch);
}

struct Ws {
    bf16* wf[4];
    bf16* wb[4];
    bf16* act[7];
};

Ws carve(void* ws, int N, int batch)
{
    Ws w{};
    bf16* p = static_cast<bf16*>(ws);
    for (int k = 0; k < 4; ++k) { w.wf[k] = p; p += kC * kK; }
    for (int k = 0; k < 4; ++k) { w.wb[k] = p; p += kC * kK; }
    const size_t a = (size_t)batch * N * N * kC;
    for (int k = 0; k < 7; ++k) { w.act[k] = p; p += a; }
    return w;
}

constexpr int kMaxCnnDevices = 64;

template <bool BIAS, bool RELU, bool MASK>
cudaError_t launch_conv32(const bf16* in, const bf16* wt, const float* bias, const bf16* mask,
                          bf16* out, int N, int batch, int sms, cudaStream_t st)
{
    // the shared-memory opt-in is per device: done once for each device this runs on
    static std::mutex lock;
    static bool done[kMaxCnnDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxCnnDevices) return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> g(lock);
        if (!done[dev]) {
            e = cudaFuncSetAttribute(cnn_conv32_kernel<BIAS, RELU, MASK>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kConvSmem);
            if (e != cudaSuccess) return e;
            done[dev] = true;
        }
    }
    const long long tiles = (long long)(N / kT2) * (N / kT2) * batch;
    const int grid = (int)(tiles < 3LL * sms ? tiles : 3LL * sms);
    cnn_conv32_kernel<BIAS, RELU, MASK><<<grid, 256, kConvSmem, st>>>(in, wt, bias, mask, out, N, batch);
    return cudaGetLastError();
}

int device_sms()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return sms;
}

cudaError_t forward(const float* params, const float* x, float* y, void* ws, int N, int batch,
                    int save, cudaStream_t st)
{
    Ws w = carve(ws, N, batch);
    for (int k = 0; k < 4; ++k)
        cnn_prep_weights_kernel<<<(kC * kC * kTaps + 255) / 256, 256, 0, st>>>(
            params + param_offset(k + 1), w.wf[k], w.wb[k]);
    const dim3 pg((N * N + 255) / 256, batch);
    // h1 .. h5 in act[0..4] when saving for the backward pass, else ping-pong in act[0..1]
    auto hbuf = [&](int k) { return save ? w.act[k] : w.act[k & 1]; };
    cnn_first_kernel<<<pg, 256, 0, st>>>(x, params, params + kC * kTaps, hbuf(0), N);
    const int sms = device_sms();
    if (sms <= 0) return cudaErrorInvalidDevice;
    for (int k = 1; k <= 4; ++k) {
        const float* b = params + param_offset(k) + (size_t)kC * kC * kTaps;
        const cudaError_t e = launch_conv32<true, true, false>(hbuf(k - 1), w.wf[k - 1], b,
                                                               nullptr, hbuf(k), N, batch, sms, st);
        if (e != cudaSuccess) return e;
    }
    cnn_last_kernel<<<pg, 256, 0, st>>>(x, hbuf(4), params + param_offset(5), y, N);
    return cudaGetLastError();
}

cudaError_t backward(const float* params, const float* x, const float* gy, float* gparams,
                     void* ws, int N, int batch, int sms, cudaStream_t st)
{
    Ws w = carve(ws, N, batch);
    cudaError_t e = cudaMemsetAsync(gparams, 0, param_count() * sizeof(float), st);
    if (e != cudaSuccess) return e;
    const dim3 pg((N * N + 255) / 256, batch);
    const int wgrid = 2 * sms;
    bf16* g[2] = {w.act[5], w.act[6]};
    // layer 6 (32 -> 1): weights from h5 and gy; gradient into z5
    float* gw = gparams + param_offset(5);
    cnn_wgrad_kernel<1, kC><<<wgrid, 256, 0, st>>>(gy, w.act[4], gw, gw + kC * kTaps, N, batch);
    cnn_last_backward_kernel<<<pg, 256, 0, st>>>(gy, w.act[4], params + param_offset(5), g[0], N);
    int cur = 0;
    // layers 5 .. 2 (32 -> 32): weights from h_{k-1} and g_z_k; gradient into z_{k-1}
    for (int k = 4; k >= 1; --k) {
        gw = gparams + param_offset(k);
        cnn_wgrad_kernel<kC, kC><<<wgrid, 256, 0, st>>>(g[cur], w.act[k - 1], gw,
                                                        gw + kC * kC * kTaps, N, batch);
        e = launch_conv32<false, false, true>(g[cur], w.wb[k - 1], nullptr, w.act[k - 1],
                                              g[cur ^ 1], N, batch, sms, st);
        if (e != cudaSuccess) return e;
        cur ^= 1;
    }
    // layer 1 (1 -> 32): weights from x and g_z1
    gw = gparams;
    cnn_wgrad_kernel<kC, 1><<<wgrid, 256, 0, st>>>(g[cur], x, gw, gw + kC * kTaps, N, batch);
    return cudaGetLastError();
}

}  // namespace cnn
}  // namespace fbp

// ---------------------------------------------------------------- C ABI
namespace {

bool cnn_aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

fbp_status cnn_check(int N, int batch)
{
    if (N < 16 || N > 4096 || (N & (N - 1)) != 0) return FBP_ERR_UNSUPPORTED;
    if (batch < 1 || batch > 65535) return FBP_ERR_INVALID_ARG;
    return FBP_OK;
}

}  // namespace

extern "C" {

size_t fbp_cnn_param_count(void) { return fbp::cnn::param_count(); }

size_t fbp_cnn_workspace_bytes(int N, int batch, int train)
{
    if (cnn_check(N, batch) != FBP_OK) return 0;
    return fbp::cnn::workspace_bytes(N, batch, train);
}

fbp_status fbp_cnn_forward(const float* d_params, const float* d_x, float* d_y, void* d_ws,
                           size_t ws_bytes, int N, int batch, int train, void* stream)
{
    fbp_status s = cnn_check(N, batch);
    if (s != FBP_OK) return s;
    if (!d_params || !d_x || !d_y || !d_ws) return FBP_ERR_INVALID_ARG;
    if (ws_bytes < fbp::cnn::workspace_bytes(N, batch, train)) return FBP_ERR_INVALID_ARG;
    if (!cnn_aligned16(d_params) || !cnn_aligned16(d_x) || !cnn_aligned16(d_y) ||
        !cnn_aligned16(d_ws))
        return FBP_ERR_MISALIGNED;
    return fbp::cnn::forward(d_params, d_x, d_y, d_ws, N, batch, train,
                             (cudaStream_t)stream) == cudaSuccess ? FBP_OK : FBP_ERR_CUDA;
}

fbp_status fbp_cnn_backward(const float* d_params, const float* d_x, const float* d_gy,
                            float* d_gparams, void* d_ws, size_t ws_bytes, int N, int batch,
                            void* stream)
{
    fbp_status s = cnn_check(N, batch);
    if (s != FBP_OK) return s;
    if (!d_params || !d_x || !d_gy || !d_gparams || !d_ws) return FBP_ERR_INVALID_ARG;
    if (ws_bytes < fbp::cnn::workspace_bytes(N, batch, 1)) return FBP_ERR_INVALID_ARG;
    if (!cnn_aligned16(d_params) || !cnn_aligned16(d_x) || !cnn_aligned16(d_gy) ||
        !cnn_aligned16(d_gparams) || !cnn_aligned16(d_ws))
        return FBP_ERR_MISALIGNED;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FBP_ERR_CUDA;
    return fbp::cnn::backward(d_params, d_x, d_gy, d_gparams, d_ws, N, batch, sms,
                              (cudaStream_t)stream) == cudaSuccess ? FBP_OK : FBP_ERR_CUDA;
}

}  // extern "C"
