// Learned residual corrector after the fast reconstruction: six 3x3 convolutions
// (1 -> 32 -> 32 -> 32 -> 32 -> 32 -> 1 channels, ReLU between, zero padding) whose output
// is added to the input image, y = x + net(x); forward and gradients for training.
//
// Hidden activation layout ("records"): bf16, per image four planes of 8 channels each
// (plane p holds channels 8p .. 8p+7, one pixel's 8 channels = one 16-byte record).  A plane
// is a zero-padded raster of (N+2) x (N+2) records -- pixel (y, x), y, x in [-1, N], at record
// kRecGuard + (y+1)(N+2) + (x+1) -- with kRecGuard zero records before it and a zero tail after.
// Every record that is not an image pixel is zero, so a 3x3 tap never needs a bounds test.
//
// The four 32 -> 32 layers run on the tcgen05 tensor cores as implicit GEMMs over the padded
// raster.  An output tile is 128 consecutive records of one image (about 128 / (N+2) rows,
// straddling row ends: pad records are computed and written back as zero).  For tap (dy,dx)
// the A operand is the 128 records starting dx records after the start of "run" dy, the
// 130 records from (tile start) + (dy-1)(N+2) - 1: three runs per plane cover all nine taps.
// A run is one contiguous 2080-byte bulk copy, and in shared memory a run of one plane is a
// stack of 8-row x 16-byte core matrices, i.e. the canonical K-major no-swizzle layout with
// the 8-row group stride (SBO) 128 bytes and the K-chunk stride (LBO) the 2080 bytes between
// the planes' copies of that run.  So every tap and every 16-channel K step is one
// tcgen05.mma (M = 128 records, N = 32 output channels, K = 16) whose A descriptor is just
// an address offset: 18 MMAs per tile, accumulating in TMEM (fp32, 32 columns per tile,
// two tiles double-buffered).  The layer's weights (32 x 288 bf16, 18 KB) are one bulk copy
// per CTA in the same layout (K chunk = tap x 4 + plane, 512 bytes apart).
//
// CTA roles (persistent, one CTA per SM): warp 0 lane 0 issues the bulk copies of each
// tile's 12 runs into a 6-stage ring (mbarrier with transaction bytes); warp 1 owns the TMEM
// allocation and its lane 0 issues the MMAs and commits them to the stage's "empty" and the
// accumulator's "full" barriers; two epilogue warpgroups (warps 2-5 and 6-9, each warp one
// TMEM lane quarter) take alternate tiles from four accumulators, read them with
// tcgen05.ld, add bias, apply ReLU or the backward mask, and store the tile's four planes as
// 16-byte records (zero for pad records).  Every wait is bounded
// (about a second); on expiry the CTA sets the corrector's status word, the other roles
// leave their loops, outstanding copies and MMAs are waited for, and TMEM is freed.
//
// The 1 -> 32 and 32 -> 1 layers, the last layer's gradient and the weight gradients run on
// the CUDA cores in fp32.  The data gradient of a 32 -> 32 layer is the same tensor-core
// kernel with the layer's weights transposed (input and output channels swapped, taps
// mirrored) and the previous layer's ReLU applied as a mask.
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
constexpr int kPlanes = kC / 8;   // 16-byte records per pixel
constexpr int kRecGuard = 8;         // zero records before the padded raster
constexpr int kTileM = 128;       // records per tensor-core tile (MMA M)
constexpr int kRun = kTileM + 2;  // records per run (tile plus the two horizontal taps)
constexpr int kRunBytes = kRun * 16;
constexpr int kStageBytes = 3 * kPlanes * kRunBytes;       // 24960
constexpr int kStages = 6;
constexpr int kWChunks = kTaps * kPlanes;                  // 36 K chunks of 8
constexpr int kWBytes = kWChunks * kC * 16;                // 18432
constexpr int kAcc = 4;           // TMEM accumulators (32 columns each)
constexpr int kEpiGroups = 2;     // epilogue warpgroups; group g takes the tiles i = g mod 2
constexpr int kConvThreads = 64 + 128 * kEpiGroups;
constexpr int kBarriers = 2 * kStages + 2 * kAcc + 2;
constexpr size_t kConvSmem = (size_t)kWBytes + (size_t)kStages * kStageBytes + kBarriers * 8 + 16;
constexpr int kTileY = 8, kTileX = 16;           // pixels per tile of the weight-gradient kernel
constexpr int kHaloY = kTileY + 2, kHaloX = kTileX + 2;

using bf16 = __nv_bfloat16;

__device__ int g_cnn_status;       // FBP_ERR_TIMEOUT after an expired wait, else 0

// Geometry of the record layout for N x N images.
struct ActGeom {
    int N, W, T;                  // image size, padded row length, tensor-core tiles per image
    long long plane;              // records per plane
};

__host__ __device__ inline ActGeom act_geom(int N)
{
    ActGeom g;
    g.N = N;
    g.W = N + 2;
    g.T = (int)(((long long)N * g.W + kTileM - 1) / kTileM);
    const long long need = kRecGuard + 2LL * g.W + (long long)kTileM * g.T + 8;
    g.plane = (need + 7) & ~7LL;
    return g;
}

__host__ __device__ inline long long rec_index(const ActGeom& g, int y, int x)
{
    return kRecGuard + (long long)(y + 1) * g.W + (x + 1);
}

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}

constexpr uint64_t kWaitNs = 1000000000ull;       // one second

// Waits for the phase of `bar` with the given parity.  Gives up when another role of the
// CTA has aborted (returns false) or after kWaitNs (sets the status word and the abort flag).
__device__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort_flag)
{
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (unsigned it = 1;; ++it) {
        if (mbar_test(bar, parity)) return true;
        if ((it & 31u) == 0) {
            if (*abort_flag) return false;
            if (global_ns() - t0 > kWaitNs) {
                *abort_flag = 1;
                atomicCAS(&g_cnn_status, 0, (int)FBP_ERR_TIMEOUT);
                return false;
            }
        }
    }
}

// The same without the abort flag, for draining work already in flight before exit.
__device__ void drain_bar(uint64_t* bar, uint32_t parity)
{
    const uint64_t t0 = global_ns();
    while (!mbar_test(bar, parity))
        if (global_ns() - t0 > kWaitNs) {
            atomicCAS(&g_cnn_status, 0, (int)FBP_ERR_TIMEOUT);
            return;
        }
}

// 1-D bulk copy global -> shared, completing `bytes` transaction bytes on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: canonical K-major layout without swizzle; lbo = byte
// stride between core matrices along K, sbo = between 8-row groups along M (or N).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: fp32 accumulator, bf16 A and B, both K-major,
// N = 32, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kC >> 3) << 17) |
                            ((uint32_t)(kTileM >> 4) << 24);

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t acc)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                 ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                   "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                   "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]),
                   "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
                   "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
                   "=r"(v[30]), "=r"(v[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 q = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&q);
}

__device__ __forceinline__ void unpack_record(const uint4 r, float* v)
{
    const uint32_t u[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u[k]));
        v[2 * k] = f.x;
        v[2 * k + 1] = f.y;
    }
}

// ---------------------------------------------------------------- weight preparation
// fp32 [co][ci][3][3] of a 32 -> 32 layer -> the shared-memory image of the GEMM's B operand:
// K chunk c = tap * 4 + (input channel / 8), then output channel, then input channel % 8.
// Forward: output channel co, input ci, tap.  Data gradient (transposed convolution): output
// channel ci, input co, tap 8 - tap.
__global__ void cnn_prep_weights_kernel(const float* __restrict__ w, bf16* __restrict__ fwd,
                                        bf16* __restrict__ bwd)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;      // co, ci, tap
    if (e >= kC * kC * kTaps) return;
    const int tap = e % kTaps;
    const int ci = (e / kTaps) % kC;
    const int co = e / (kTaps * kC);
    const bf16 v = __float2bfloat16_rn(w[e]);
    fwd[((tap * kPlanes + ci / 8) * kC + co) * 8 + ci % 8] = v;
    const int mt = kTaps - 1 - tap;
    bwd[((mt * kPlanes + co / 8) * kC + ci) * 8 + co % 8] = v;
}

// ---------------------------------------------------------------- 32 -> 32 on tcgen05
struct ConvArgs {
    const uint4* in;        // records of `images` images
    const bf16* wimg;       // weight image (kWBytes)
    const float* bias;      // [32] (BIAS)
    const uint4* mask;      // records (MASK): output channel c kept where mask's c > 0
    uint4* out;             // records
    int N, images;
};

template <bool BIAS, bool RELU, bool MASK>
__global__ void __launch_bounds__(kConvThreads, 1)
cnn_conv32_kernel(ConvArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* wsm = smem;
    unsigned char* stages = smem + kWBytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(stages + (size_t)kStages * kStageBytes);
    uint64_t* full = bars;                  // [kStages] runs landed
    uint64_t* empty = bars + kStages;       // [kStages] runs consumed by the MMAs
    uint64_t* tfull = bars + 2 * kStages;   // [kAcc] accumulator complete
    uint64_t* tempty = tfull + kAcc;        // [kAcc] accumulator read out
    uint64_t* wbar = tempty + kAcc;         // weights landed
    uint64_t* drain = wbar + 1;             // MMAs of this CTA complete (exit)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const ActGeom G = act_geom(a.N);
    const long long total = (long long)G.T * a.images;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        for (int b = 0; b < kAcc; ++b) {
            mbar_init(tfull + b, 1);
            mbar_init(tempty + b, 4);
        }
        mbar_init(wbar, 1);
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "n"(kAcc * kC) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---- producer: weights once, then the 12 runs of every tile
            mbar_expect_tx(wbar, kWBytes);
            bulk_g2s(wsm, a.wimg, kWBytes, wbar);
            long long i = 0;
            int img = (int)(blockIdx.x / G.T), tt = (int)(blockIdx.x % G.T);
            for (long long t = blockIdx.x; t < total; t += gridDim.x, ++i) {
                const int s = (int)(i % kStages);
                const uint32_t k = (uint32_t)(i / kStages);
                if (i > 0) {                               // next tile of this CTA
                    tt += gridDim.x;
                    while (tt >= G.T) { tt -= G.T; ++img; }
                }
                if (!wait_bar(empty + s, (k & 1u) ^ 1u, abort_flag)) break;
                const long long m0 = kRecGuard + G.W + (long long)kTileM * tt;
                mbar_expect_tx(full + s, kStageBytes);
                unsigned char* dst = stages + (size_t)s * kStageBytes;
#pragma unroll 1
                for (int dy = 0; dy < 3; ++dy)
#pragma unroll 1
                    for (int p = 0; p < kPlanes; ++p) {
                        const uint4* src = a.in + ((long long)img * kPlanes + p) * G.plane + m0 +
                                           (long long)(dy - 1) * G.W - 1;
                        bulk_g2s(dst + (dy * kPlanes + p) * kRunBytes, src, kRunBytes, full + s);
                    }
            }
            // copies still in flight land before the CTA exits
            for (long long j = i - kStages; j < i; ++j)
                if (j >= 0) drain_bar(full + (int)(j % kStages), (uint32_t)(j / kStages) & 1u);
            drain_bar(wbar, 0);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer
            if (wait_bar(wbar, 0, abort_flag)) {
                tc_fence_after();
                const uint32_t wbase = smem_u32(wsm);
                const uint32_t sbase = smem_u32(stages);
                long long i = 0;
                for (long long t = blockIdx.x; t < total; t += gridDim.x, ++i) {
                    const int s = (int)(i % kStages);
                    const uint32_t k = (uint32_t)(i / kStages);
                    const int b = (int)(i % kAcc);
                    const uint32_t j = (uint32_t)(i / kAcc);
                    if (!wait_bar(full + s, k & 1u, abort_flag)) break;
                    if (!wait_bar(tempty + b, (j & 1u) ^ 1u, abort_flag)) break;
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(b * kC);
                    const uint32_t abase = sbase + (uint32_t)(s * kStageBytes);
#pragma unroll
                    for (int tap = 0; tap < kTaps; ++tap) {
                        const int dy = tap / 3, dx = tap % 3;
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
                            const uint32_t aa = abase + (uint32_t)((dy * kPlanes + 2 * kk) * kRunBytes + dx * 16);
                            const uint32_t ba = wbase + (uint32_t)((tap * kPlanes + 2 * kk) * kC * 16);
                            umma(d, smem_desc(aa, kRunBytes, 128), smem_desc(ba, kC * 16, 128),
                                 (tap | kk) != 0 ? 1u : 0u);
                        }
                    }
                    umma_commit(empty + s);
                    umma_commit(tfull + b);
                }
            }
            umma_commit(drain);                 // everything issued above has completed ...
            drain_bar(drain, 0);                // ... once this phase does
        }
    } else {
        // ---- epilogue: warpgroup eg (warps 2+4eg .. 5+4eg) takes tiles i = eg mod 2; each
        // warp reads TMEM lane quarter warp % 4
        const int q = warp & 3;
        const int row = 32 * q + lane;
        const int eg = (warp - 2) >> 2;
        const int etid = threadIdx.x - 64;               // 0 .. 128 kEpiGroups - 1
        // zero the records no tile writes: the guard and top pad row, and the tail
        const long long head = kRecGuard + G.W;
        const long long tail0 = kRecGuard + G.W + (long long)kTileM * G.T;
        const long long tail = G.plane - tail0;
        const long long nz = (long long)a.images * kPlanes * (head + tail);
        for (long long z = (long long)blockIdx.x * (128 * kEpiGroups) + etid; z < nz;
             z += (long long)gridDim.x * (128 * kEpiGroups)) {
            const long long pl = z / (head + tail);
            const long long r = z - pl * (head + tail);
            a.out[pl * G.plane + (r < head ? r : tail0 + (r - head))] = make_uint4(0u, 0u, 0u, 0u);
        }
        float bias[kC];
#pragma unroll
        for (int c = 0; c < kC; ++c) bias[c] = BIAS ? __ldg(a.bias + c) : 0.0f;
        long long i = eg;
        int img = (int)((blockIdx.x + (long long)eg * gridDim.x) / G.T);
        int tt = (int)((blockIdx.x + (long long)eg * gridDim.x) % G.T);
        const int step = kEpiGroups * gridDim.x;
        for (long long t = blockIdx.x + (long long)eg * gridDim.x; t < total;
             t += step, i += kEpiGroups) {
            if (i != eg) {                               // next tile of this warpgroup
                tt += step;
                while (tt >= G.T) { tt -= G.T; ++img; }
            }
            const int b = (int)(i % kAcc);
            const uint32_t j = (uint32_t)(i / kAcc);
            if (!wait_bar(tfull + b, j & 1u, abort_flag)) break;
            tc_fence_after();
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * kC), v);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty + b);
            // pixel of this record: 32-bit arithmetic (a plane has < 2^31 records)
            const unsigned rel = (unsigned)(G.W + kTileM * tt + row);
            const unsigned yy = rel / (unsigned)G.W;
            const int y = (int)yy - 1;
            const int x = (int)(rel - yy * (unsigned)G.W) - 1;
            const long long m = kRecGuard + (long long)rel;
            const bool inside = (unsigned)y < (unsigned)a.N && (unsigned)x < (unsigned)a.N;
            float mk[kC];
            if (MASK && inside) {
#pragma unroll
                for (int p = 0; p < kPlanes; ++p)
                    unpack_record(a.mask[((long long)img * kPlanes + p) * G.plane + m], mk + 8 * p);
            }
#pragma unroll
            for (int p = 0; p < kPlanes; ++p) {
                uint32_t w4[4];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int c = 8 * p + 2 * h;
                    float v0 = __uint_as_float(v[c]), v1 = __uint_as_float(v[c + 1]);
                    if (BIAS) { v0 += bias[c]; v1 += bias[c + 1]; }
                    if (RELU) { v0 = fmaxf(v0, 0.0f); v1 = fmaxf(v1, 0.0f); }
                    if (MASK) {
                        v0 = mk[c] > 0.0f ? v0 : 0.0f;
                        v1 = mk[c + 1] > 0.0f ? v1 : 0.0f;
                    }
                    w4[h] = inside ? pack_bf16(v0, v1) : 0u;
                }
                a.out[((long long)img * kPlanes + p) * G.plane + m] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(kAcc * kC) : "memory");
    }
}

// ---------------------------------------------------------------- 1 -> 32 and 32 -> 1
// First layer: h[p][o] = relu(b[o] + sum_tap w[o][tap] x[p + off(tap)]), fp32 math, written
// as records over the whole plane (zero outside the image).  The weights sit in shared
// memory as [tap][o] and reach registers as 16-byte broadcasts, 32 per tap; each thread
// computes the records r and r + kFirstStride.
constexpr int kFirstStride = 128;           // records between a thread's two records
__global__ void __launch_bounds__(128)
cnn_first_kernel(const float* __restrict__ x, const float* __restrict__ w,
                 uint4* __restrict__ h, int N)
{
    __shared__ __align__(16) float ws[kTaps][kC];
    __shared__ float bs[kC];
    for (int e = threadIdx.x; e < kC * kTaps; e += blockDim.x) ws[e % kTaps][e / kTaps] = w[e];
    for (int e = threadIdx.x; e < kC; e += blockDim.x) bs[e] = w[kC * kTaps + e];
    __syncthreads();
    const ActGeom G = act_geom(N);
    const long long r0 = (long long)blockIdx.x * 2 * kFirstStride + threadIdx.x;
    const int img = blockIdx.y;
    const float* xs = x + (size_t)img * N * N;
    float v[2][kTaps];
    bool inside[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const long long r = r0 + u * kFirstStride;
        int py = -2, px = -2;                   // pixel of record r (32-bit: r < 2^31)
        if (r >= kRecGuard && r < G.plane) {
            const unsigned q = (unsigned)(r - kRecGuard);
            const unsigned yy = q / (unsigned)G.W;
            py = (int)yy - 1;
            px = (int)(q - yy * (unsigned)G.W) - 1;
        }
        inside[u] = (unsigned)py < (unsigned)N && (unsigned)px < (unsigned)N;
#pragma unroll
        for (int tap = 0; tap < kTaps; ++tap) {
            const int yy = py + tap / 3 - 1, xx = px + tap % 3 - 1;
            v[u][tap] = (inside[u] && yy >= 0 && yy < N && xx >= 0 && xx < N) ? xs[(size_t)yy * N + xx] : 0.0f;
        }
    }
    float acc[2][kC];
#pragma unroll
    for (int o = 0; o < kC; ++o) acc[0][o] = acc[1][o] = bs[o];
#pragma unroll
    for (int tap = 0; tap < kTaps; ++tap) {
#pragma unroll
        for (int o4 = 0; o4 < kC; o4 += 4) {
            const float4 wv = *reinterpret_cast<const float4*>(&ws[tap][o4]);
            const float wk[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                acc[0][o4 + k] = fmaf(wk[k], v[0][tap], acc[0][o4 + k]);
                acc[1][o4 + k] = fmaf(wk[k], v[1][tap], acc[1][o4 + k]);
            }
        }
    }
    uint4* dst = h + (long long)img * kPlanes * G.plane;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const long long r = r0 + u * kFirstStride;
        if (r >= G.plane) continue;
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) {
            uint32_t w4[4];
#pragma unroll
            for (int hh = 0; hh < 4; ++hh) {
                const int o = 8 * p + 2 * hh;
                w4[hh] = inside[u] ? pack_bf16(fmaxf(acc[u][o], 0.0f), fmaxf(acc[u][o + 1], 0.0f)) : 0u;
            }
            dst[p * G.plane + r] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
        }
    }
}

// the 32 channels of record r of one image's planes
__device__ __forceinline__ void load_pixel32(float (&v)[kC], const uint4* planes, long long plane,
                                             long long r)
{
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) unpack_record(planes[p * plane + r], v + 8 * p);
}

// Last layer and the skip connection: y[p] = x[p] + b + sum_{tap, c} w[c][tap] h[p + off][c].
// One 16 x 16 output tile per CTA: its 18 x 18 records (four planes) are staged in shared
// memory once; the weights sit there as [tap][c] and reach registers as 16-byte broadcasts;
// each thread sums the 9 taps x 32 channels of two pixels, rows ly and ly + 8 (pad records
// are zero: no bounds tests).
constexpr int kLT = 16;
constexpr int kLH = kLT + 2;
__global__ void __launch_bounds__(kLT * kLT / 2)
cnn_last_kernel(const float* __restrict__ x, const uint4* __restrict__ h, const float* __restrict__ w,
                float* __restrict__ y, int N)
{
    __shared__ __align__(16) float ws[kTaps][kC];
    __shared__ uint4 hs[kPlanes][kLH * kLH];
    for (int e = threadIdx.x; e < kC * kTaps; e += blockDim.x) ws[e % kTaps][e / kTaps] = w[e];
    const float bias = w[kC * kTaps];
    const ActGeom G = act_geom(N);
    const int tiles_x = N / kLT;
    const int y0 = (int)(blockIdx.x / tiles_x) * kLT, x0 = (int)(blockIdx.x % tiles_x) * kLT;
    const uint4* hp = h + (long long)blockIdx.y * kPlanes * G.plane;
    for (int e = threadIdx.x; e < kPlanes * kLH * kLH; e += blockDim.x) {
        const int p = e / (kLH * kLH), r = e - p * (kLH * kLH);
        const int ty = r / kLH, tx = r - ty * kLH;
        hs[p][r] = hp[p * G.plane + rec_index(G, y0 - 1 + ty, x0 - 1 + tx)];
    }
    __syncthreads();
    const int ly = threadIdx.x / kLT, lx = threadIdx.x % kLT;      // rows ly and ly + 8
    float s0 = bias, s1 = bias;
    for (int tap = 0; tap < kTaps; ++tap) {
        const int r = (ly + tap / 3) * kLH + lx + tap % 3;
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) {
            float v0[8], v1[8];
            unpack_record(hs[p][r], v0);
            unpack_record(hs[p][r + (kLT / 2) * kLH], v1);
            const float4 wa = *reinterpret_cast<const float4*>(&ws[tap][8 * p]);
            const float4 wb = *reinterpret_cast<const float4*>(&ws[tap][8 * p + 4]);
            const float wk[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                s0 = fmaf(wk[e], v0[e], s0);
                s1 = fmaf(wk[e], v1[e], s1);
            }
        }
    }
    const size_t pix = (size_t)blockIdx.y * N * N + (size_t)(y0 + ly) * N + x0 + lx;
    y[pix] = x[pix] + s0;
    const size_t pix1 = pix + (size_t)(kLT / 2) * N;
    y[pix1] = x[pix1] + s1;
}

// Gradient through the last layer into the fifth layer's pre-activation:
// g[p][c] = (h5[p][c] > 0) * sum_tap w[c][tap] gy[p - off(tap)], as records over the whole
// plane (zero outside the image).
__global__ void __launch_bounds__(256)
cnn_last_backward_kernel(const float* __restrict__ gy, const uint4* __restrict__ h5,
                         const float* __restrict__ w, uint4* __restrict__ g, int N)
{
    __shared__ float ws[kC * kTaps];
    for (int e = threadIdx.x; e < kC * kTaps; e += blockDim.x) ws[e] = w[e];
    __syncthreads();
    const ActGeom G = act_geom(N);
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= G.plane) return;
    int py = -2, px = -2;                       // pixel of record r (32-bit: r < 2^31)
    if (r >= kRecGuard) {
        const unsigned u = (unsigned)(r - kRecGuard);
        const unsigned yy = u / (unsigned)G.W;
        py = (int)yy - 1;
        px = (int)(u - yy * (unsigned)G.W) - 1;
    }
    const long long ib = (long long)blockIdx.y * kPlanes * G.plane;
    uint4* dst = g + ib + r;
    if ((unsigned)py >= (unsigned)N || (unsigned)px >= (unsigned)N) {
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) dst[p * G.plane] = make_uint4(0u, 0u, 0u, 0u);
        return;
    }
    const size_t img = (size_t)blockIdx.y * N * N;
    float v[kTaps];
#pragma unroll
    for (int tap = 0; tap < kTaps; ++tap) {
        const int yy = py - (tap / 3 - 1), xx = px - (tap % 3 - 1);
        v[tap] = (yy >= 0 && yy < N && xx >= 0 && xx < N) ? gy[img + (size_t)yy * N + xx] : 0.0f;
    }
    float m[kC];
    load_pixel32(m, h5 + ib, G.plane, r);
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) {
        uint32_t w4[4];
#pragma unroll
        for (int hh = 0; hh < 4; ++hh) {
            const int c = 8 * p + 2 * hh;
            float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
            for (int tap = 0; tap < kTaps; ++tap) {
                s0 = fmaf(ws[c * kTaps + tap], v[tap], s0);
                s1 = fmaf(ws[(c + 1) * kTaps + tap], v[tap], s1);
            }
            w4[hh] = pack_bf16(m[c] > 0.0f ? s0 : 0.0f, m[c + 1] > 0.0f ? s1 : 0.0f);
        }
        dst[p * G.plane] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
    }
}

// ---------------------------------------------------------------- weight gradients (fp32)
// gw[o][c][tap] += sum_p gz[p][o] hp[p + off(tap)][c], gb[o] += sum_p gz[p][o], over all pixels
// of all images.  CO / CI are 32 or 1; a 1-channel operand is fp32 [N][N] (the image or the
// output gradient), a 32-channel one records.  Persistent CTAs accumulate over 8 x 16-pixel
// tiles in registers and add once into the global gradient.
__device__ __forceinline__ float record_channel(const uint4* planes, long long plane, long long r, int c)
{
    const bf16* rec = reinterpret_cast<const bf16*>(planes + (c >> 3) * plane + r);
    return __bfloat162float(rec[c & 7]);
}

template <int CO, int CI>
__global__ void __launch_bounds__(256)
cnn_wgrad_kernel(const void* __restrict__ gz_, const void* __restrict__ hp_, float* __restrict__ gw,
                 float* __restrict__ gb, int N, int images)
{
    constexpr int NOUT = CO * CI * kTaps;
    constexpr int PER = (NOUT + 255) / 256;
    __shared__ float gzs[kTileY * kTileX][CO];
    __shared__ float hps[kHaloY * kHaloX][CI];
    const ActGeom G = act_geom(N);
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
        const long long ib = (long long)im * kPlanes * G.plane;
        __syncthreads();                               // previous tile consumed
        for (int e = tid; e < kTileY * kTileX * CO; e += 256) {
            const int pix = e / CO, o = e - pix * CO;
            const int yy = y0 + pix / kTileX, xx = x0 + pix % kTileX;
            gzs[pix][o] = CO == 1 ? static_cast<const float*>(gz_)[img + (size_t)yy * N + xx]
                                  : record_channel(static_cast<const uint4*>(gz_) + ib, G.plane,
                                                   rec_index(G, yy, xx), o);
        }
        for (int e = tid; e < kHaloY * kHaloX * CI; e += 256) {
            const int pix = e / CI, c = e - pix * CI;
            const int gy = y0 - 1 + pix / kHaloX, gx = x0 - 1 + pix % kHaloX;
            float v = 0.0f;
            if (CI == 1) {
                if (gy >= 0 && gy < N && gx >= 0 && gx < N)
                    v = static_cast<const float*>(hp_)[img + (size_t)gy * N + gx];
            } else {
                v = record_channel(static_cast<const uint4*>(hp_) + ib, G.plane, rec_index(G, gy, gx), c);
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

size_t act_bytes(int N, int batch) { return (size_t)batch * kPlanes * act_geom(N).plane * 16; }

// workspace: the weight images (4 layers x forward and transposed), then `nbuf` record
// buffers (5 activations and 2 gradients when training, a ping-pong pair otherwise)
size_t workspace_bytes(int N, int batch, int train)
{
    const size_t wbytes = (size_t)4 * 2 * kWBytes;
    const int nbuf = train ? 5 + 2 : 2;
    return wbytes + (size_t)nbuf * act_bytes(N, batch);
}

struct Ws {
    bf16* wf[4];
    bf16* wb[4];
    uint4* act[7];
};

Ws carve(void* ws, int N, int batch, int train)
{
    Ws w{};
    unsigned char* p = static_cast<unsigned char*>(ws);
    for (int k = 0; k < 4; ++k) { w.wf[k] = reinterpret_cast<bf16*>(p); p += kWBytes; }
    for (int k = 0; k < 4; ++k) { w.wb[k] = reinterpret_cast<bf16*>(p); p += kWBytes; }
    const size_t a = act_bytes(N, batch);
    for (int k = 0; k < (train ? 7 : 2); ++k) { w.act[k] = reinterpret_cast<uint4*>(p); p += a; }
    return w;
}

constexpr int kMaxCnnDevices = 64;

template <bool BIAS, bool RELU, bool MASK>
cudaError_t launch_conv32(const uint4* in, const bf16* wt, const float* bias, const uint4* mask,
                          uint4* out, int N, int batch, int sms, cudaStream_t st)
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
    const long long tiles = (long long)act_geom(N).T * batch;
    const int grid = (int)(tiles < sms ? tiles : sms);
    ConvArgs a{in, wt, bias, mask, out, N, batch};
    cnn_conv32_kernel<BIAS, RELU, MASK><<<grid, kConvThreads, kConvSmem, st>>>(a);
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
    Ws w = carve(ws, N, batch, save);
    for (int k = 0; k < 4; ++k)
        cnn_prep_weights_kernel<<<(kC * kC * kTaps + 255) / 256, 256, 0, st>>>(
            params + param_offset(k + 1), w.wf[k], w.wb[k]);
    const ActGeom G = act_geom(N);
    const dim3 fg((unsigned)((G.plane + 2 * kFirstStride - 1) / (2 * kFirstStride)), batch);
    const dim3 lg((N / kLT) * (N / kLT), batch);
    // h1 .. h5 in act[0..4] when saving for the backward pass, else ping-pong in act[0..1]
    auto hbuf = [&](int k) { return save ? w.act[k] : w.act[k & 1]; };
    cnn_first_kernel<<<fg, 128, 0, st>>>(x, params, hbuf(0), N);
    const int sms = device_sms();
    if (sms <= 0) return cudaErrorInvalidDevice;
    for (int k = 1; k <= 4; ++k) {
        const float* b = params + param_offset(k) + (size_t)kC * kC * kTaps;
        const cudaError_t e = launch_conv32<true, true, false>(hbuf(k - 1), w.wf[k - 1], b,
                                                               nullptr, hbuf(k), N, batch, sms, st);
        if (e != cudaSuccess) return e;
    }
    cnn_last_kernel<<<lg, kLT * kLT / 2, 0, st>>>(x, hbuf(4), params + param_offset(5), y, N);
    return cudaGetLastError();
}

cudaError_t backward(const float* params, const float* x, const float* gy, float* gparams,
                     void* ws, int N, int batch, int sms, cudaStream_t st)
{
    Ws w = carve(ws, N, batch, 1);
    cudaError_t e = cudaMemsetAsync(gparams, 0, param_count() * sizeof(float), st);
    if (e != cudaSuccess) return e;
    const ActGeom G = act_geom(N);
    const dim3 rg((unsigned)((G.plane + 255) / 256), batch);
    const int wgrid = 2 * sms;
    uint4* g[2] = {w.act[5], w.act[6]};
    // layer 6 (32 -> 1): weights from h5 and gy; gradient into z5
    float* gw = gparams + param_offset(5);
    cnn_wgrad_kernel<1, kC><<<wgrid, 256, 0, st>>>(gy, w.act[4], gw, gw + kC * kTaps, N, batch);
    cnn_last_backward_kernel<<<rg, 256, 0, st>>>(gy, w.act[4], params + param_offset(5), g[0], N);
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

fbp_status fbp_cnn_last_error(void)
{
    if (cudaDeviceSynchronize() != cudaSuccess) return FBP_ERR_CUDA;
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, fbp::g_cnn_status, sizeof(int)) != cudaSuccess) return FBP_ERR_CUDA;
    if (v != 0) {
        const int zero = 0;
        if (cudaMemcpyToSymbol(fbp::g_cnn_status, &zero, sizeof(int)) != cudaSuccess) return FBP_ERR_CUDA;
    }
    return (fbp_status)v;
}

}  // extern "C"
