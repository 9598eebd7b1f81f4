// Learned residual corrector after the fast reconstruction: six 3x3 convolutions
// (1 -> 32 -> 32 -> 32 -> 32 -> 32 -> 1 channels, ReLU between, zero padding) whose output
// is added to the input image, y = x + net(x); forward and gradients for training.
//
// Hidden activation layout ("records"): bf16, one 64-byte record per pixel holding its 32
// channels, the record's four 16-byte chunks (channels 8c .. 8c+7) stored XOR-permuted:
// chunk c of record r at chunk position c ^ ((r >> 1) & 3) -- the 64-byte swizzle of the
// tensor cores' shared-memory operands, applied in global memory already.  An image is a
// zero-padded raster of (N+2) x (N+2) records -- pixel (y, x), y, x in [-1, N], at record
// kRecGuard + (y+1)(N+2) + (x+1) -- with kRecGuard zero records before it and a zero tail
// after.  Every record that is not an image pixel is zero, so a 3x3 tap never needs a
// bounds test.
//
// The four 32 -> 32 layers run on the tcgen05 tensor cores as implicit GEMMs over the padded
// raster, with the pixels as the MMA's N dimension: an MMA costs about the same up to
// N = 128 whatever its width, so each one should carry as many pixels as it can.  An output
// tile is 254 consecutive records of one image (straddling row ends: pad records are
// computed and written back as zero).  "Run" dy is the 256 records from (tile start) +
// (dy-1)(N+2) - 1, one contiguous 16-KB bulk copy placed in shared memory so that its row
// index is congruent to its record index mod 8: the records then sit exactly in the
// canonical K-major 64-byte-swizzled layout (8-row atoms of 512 bytes, row = one pixel's 32
// channels) and serve as the B operand (N = 256 rows).  The A operand (M = 128 rows) stacks
// the layer's weights for the three horizontal taps dx of one dy: row 32q + 8dx + o' holds
// output channel 8q + o' at tap (dy, dx) (rows 32q + 24 .. 32q + 31 are zero).  So one MMA
// per dy and 16-channel step, 6 per tile, accumulates D[(q, dx, o')][j] = the tile's
// contribution of tap column dx at run row j, in TMEM (fp32, 256 columns).  The output
// pixel i of the tile is D[dx = 0][i] + D[dx = 1][i + 1] + D[dx = 2][i + 2]: the epilogue
// reads TMEM with the 16x256b shape, which gives one thread the rows of taps 0 and 1 of
// one channel at the same two columns (and, from the upper 16 lanes, tap 2), so the sum
// needs the neighbouring column pair only: two warp shuffles per 8 columns.  A stmatrix
// transpose turns each warp's [channel][pixel] block into the 16-byte chunks of the pixel
// records it stores.  The weights (128 x 96 bf16 = 24 KB) are one bulk copy per CTA in the
// K-major layout without swizzle (K chunk = dy x 4 + input channel / 8, 2 KB apart).
//
// CTA roles (persistent, one CTA per SM): warp 0 lane 0 issues the bulk copies of each
// tile's 3 runs into a 3-stage ring (mbarrier with transaction bytes); warp 1 owns the TMEM
// allocation (two 256-column accumulators) and its lane 0 issues the MMAs and commits them
// to the stage's "empty" and the accumulator's "full" barriers; four epilogue warpgroups
// (warps 2-17, each warp one TMEM lane quarter) share every tile, each taking 64 of its 256
// columns, read them with tcgen05.ld, add bias, apply ReLU or the backward mask, and store
// the tile's records (zero for pad records).  Every wait is bounded (about a second); on
// expiry the CTA sets the corrector's status word, the other roles leave their loops,
// outstanding copies and MMAs are waited for, and TMEM is freed.
//
// The 32 -> 1 layer runs in the same tensor-core kernel (its fp32 weights split exactly
// into three bf16 parts, so that the products and their fp32 sums are those of the fp32
// weights).  The weight gradients of the 32 -> 32 layers are a tensor-core GEMM over the
// records (cnn_wgrad_tc_kernel).  The 1 -> 32 layer, the last layer's gradient and the
// 1-channel layers' weight gradients run on the CUDA cores in fp32.  The data gradient of a
// 32 -> 32 layer is the same tensor-core
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
constexpr int kPlanes = kC / 8;   // 16-byte chunks per pixel record
constexpr int kRecGuard = 8;      // zero records before the padded raster
constexpr int kTileOut = 254;     // output records per tensor-core tile
constexpr int kNpix = 256;        // run rows per MMA (its N)
constexpr int kRecBytes = 64;     // one pixel's 32 bf16 channels
constexpr int kRunCopy = kNpix * kRecBytes;                // 16384 bytes per run copy
constexpr int kRunBytes = 264 * kRecBytes;                 // run buffer: 7 rows of phase + 256, in atoms
constexpr int kStageBytes = 3 * kRunBytes;                 // 50688
constexpr int kStages = 3;
constexpr int kWRows = 128;                                // A rows: (lane quarter, dx, channel)
constexpr int kWChunks = 3 * kPlanes;                      // 12 K chunks of 8: (dy, input channel / 8)
constexpr int kWImgChunks = kWChunks + 2;                  // + one K step: the bias in three bf16 parts
constexpr int kWBytes = kWImgChunks * kWRows * 16;         // 28672
constexpr int kOnesBytes = 2 * kNpix * 16;                 // the bias step's B operand: all ones
constexpr int kAcc = 2;           // TMEM accumulators (256 columns each)
constexpr int kTmemCols = 512;
constexpr int kEpiGroups = 4;     // epilogue warpgroups, all sharing every tile
constexpr int kChunksPerEpi = kNpix / 32 / kEpiGroups;     // 32-column chunks per warp and tile
static_assert(kChunksPerEpi == 2, "each epilogue warp reads two chunks with one batch of loads");
constexpr int kConvThreads = 64 + 128 * kEpiGroups;
constexpr int kBarriers = 2 * kStages + 2 * kAcc + 2;
constexpr int kScratchBytes = 4 * kEpiGroups * 512;        // per epilogue warp: 32 pixels x 8 channels bf16
constexpr size_t kConvSmem = 1024 + (size_t)kWBytes + kOnesBytes + (size_t)kStages * kStageBytes + kScratchBytes +
                             kBarriers * 8 + 16;
constexpr int kTileY = 8, kTileX = 16;           // pixels per tile of the weight-gradient kernel
constexpr int kHaloY = kTileY + 2, kHaloX = kTileX + 2;

using bf16 = __nv_bfloat16;

__device__ int g_cnn_status;       // FBP_ERR_TIMEOUT after an expired wait, else 0

// Range checks of the bounds-checked build (FBP_BOUNDS_CHECK): an index outside its buffer
// records FBP_ERR_INTERNAL in the corrector's status word and the access is skipped (a
// skipped load reads 0; a skipped bulk copy leaves its stage unfilled, so the wait for it
// expires and the CTA stops).  In the normal build every check is true and compiles away.
__device__ __forceinline__ bool cnn_ok(long long i, long long n)
{
    return in_bounds(&g_cnn_status, i, n);
}

// [i, i + len) inside [0, n)
__device__ __forceinline__ bool cnn_span_ok(long long i, long long len, long long n)
{
    return cnn_ok(i, n) && cnn_ok(i + len - 1, n);
}

#ifdef FBP_BOUNDS_CHECK
// Test hook (fbp_check_cnn_image_limit): when > 0, the last layer checks its image loads and
// stores against this many images instead of the call's count.
__device__ int g_cnn_image_limit;
#endif

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
    g.T = (int)(((long long)N * g.W + kTileOut - 1) / kTileOut);
    // room for the convolution's runs and for the weight gradient's (256-record tiles,
    // runs reaching W + 256 records past a tile's start)
    const long long tw = ((long long)N * g.W + 255) / 256;
    long long need = kRecGuard + 2LL * g.W + (long long)kTileOut * g.T + 8;
    const long long need_wg = kRecGuard + 2LL * g.W + 256 * tw + 16;
    if (need_wg > need) need = need_wg;
    g.plane = (need + 7) & ~7LL;
    return g;
}

__host__ __device__ inline long long rec_index(const ActGeom& g, int y, int x)
{
    return kRecGuard + (long long)(y + 1) * g.W + (x + 1);
}

// position of chunk c (channels 8c .. 8c+7) within record r
__host__ __device__ inline int chunk_pos(long long r, int c) { return c ^ (int)((r >> 1) & 3); }

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

// One bounded wait for the phase: the thread may sleep up to kSuspendNs inside the try
// (instead of spinning through issue slots) and returns whether the phase has completed.
constexpr unsigned kSuspendNs = 100000;
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
                 " selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity), "n"(kSuspendNs) : "memory");
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

// The same for the 64-byte-swizzled K-major layout: 8-row atoms of 512 bytes (SBO), the
// swizzle taken from the address bits (a start at any 64-byte row, plus 32 bytes per K step).
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t addr)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
           (1ull << 46) | (4ull << 61);
}

// Instruction descriptor of kind::f16: fp32 accumulator, bf16 A and B, both K-major,
// N = 256 (pixels), M = 128 (weight rows).
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kNpix >> 3) << 17) |
                            ((uint32_t)(kWRows >> 4) << 24);

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t acc)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                 ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ void umma_idesc(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t acc)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                 ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)) : "memory");
}

// 16x256b shapes: thread t receives TMEM lane (base + t/4) at columns 2(t%4), 2(t%4)+1 and
// lane (base + 8 + t/4) at the same columns; each further repetition is 8 columns on.
__device__ __forceinline__ void tmem_ld16_x8(uint32_t taddr, uint32_t* v)
{
    asm volatile("tcgen05.ld.sync.aligned.16x256b.x8.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                   "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                   "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]),
                   "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
                   "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
                   "=r"(v[30]), "=r"(v[31])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld16_x2(uint32_t taddr, uint32_t* v)
{
    asm volatile("tcgen05.ld.sync.aligned.16x256b.x2.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                   "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld16_x1(uint32_t taddr, uint32_t* v)
{
    asm volatile("tcgen05.ld.sync.aligned.16x256b.x1.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]) : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld()
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Four 8 x 8 bf16 matrices, fragment of thread t = (row t / 4, columns 2(t % 4), +1), stored
// transposed: row j of matrix i (the fragment's column j) to the 16 bytes at the address
// that thread 8i + j supplies.
__device__ __forceinline__ void stmatrix_x4_trans(uint32_t addr, uint32_t r0, uint32_t r1, uint32_t r2,
                                                  uint32_t r3)
{
    asm volatile("stmatrix.sync.aligned.m8n8.x4.trans.shared.b16 [%0], {%1,%2,%3,%4};"
                 ::"r"(addr), "r"(r0), "r"(r1), "r"(r2), "r"(r3) : "memory");
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
// A float32 value as the exact sum of three bf16 values, hi = bf16(v), mid = bf16(v - hi),
// lo = bf16(v - hi - mid): after two bf16 parts at most 8 significant bits are left.
__device__ __forceinline__ float bf16_round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// part 0, 1, 2 (hi, mid, lo) of v split exactly into three bf16 values
__device__ __forceinline__ float bf16_part(float v, int part)
{
    const float hi = bf16_round(v);
    const float mid = bf16_round(v - hi);
    const float lo = bf16_round((v - hi) - mid);
    return part == 0 ? hi : (part == 1 ? mid : lo);
}

// fp32 [co][ci][3][3] of a 32 -> 32 layer -> the shared-memory image of the GEMM's A operand:
// K chunk (dy * 4 + input channel / 8), then row 32 (o / 8) + 8 dx + o % 8, then input
// channel % 8 (rows 32 q + 24 .. 32 q + 31 zero).  Forward: output o = co, input ci, tap
// (dy, dx).  Data gradient (transposed convolution): output o = ci, input co, tap
// (2 - dy, 2 - dx).  Chunks 12 and 13 are the bias step of the forward image: K column p of
// row 32q + o' (tap dx = 0) holds part p (bf16_part) of output channel 8q + o''s bias,
// multiplied by a B operand of ones; everything else there is zero.  One thread per element of the image.
__global__ void cnn_prep_weights_kernel(const float* __restrict__ w, bf16* __restrict__ fwd,
                                        bf16* __restrict__ bwd)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;      // (chunk, row, lane of 8)
    if (e >= kWImgChunks * kWRows * 8) return;
    const int c8 = e & 7;
    const int row = (e >> 3) % kWRows;
    const int chunk = e / (8 * kWRows);
    if (chunk >= kWChunks) {
        const int q = row / 32, dx = (row % 32) / 8, ol = row % 8;
        const bool part = chunk == kWChunks && dx == 0 && c8 < 3;
        const int bi = kC * kC * kTaps + 8 * q + ol;               // bias of output channel 8q + ol
        fwd[e] = __float2bfloat16_rn(part && cnn_ok(bi, kC * kC * kTaps + kC) ? bf16_part(w[bi], c8) : 0.0f);
        bwd[e] = __float2bfloat16_rn(0.0f);
        return;
    }
    const int dy = chunk / kPlanes, cin = (chunk % kPlanes) * 8 + c8;
    const int q = row / 32, dx = (row % 32) / 8, ol = row % 8;
    const int o = 8 * q + ol;
    float vf = 0.0f, vb = 0.0f;
    if (dx < 3) {
        const int fi = ((o * kC + cin) * 3 + dy) * 3 + dx;              // W[o][cin][dy][dx]
        const int bi = ((cin * kC + o) * 3 + (2 - dy)) * 3 + (2 - dx);  // W[cin][o][2-dy][2-dx]
        if (cnn_ok(fi, kC * kC * kTaps)) vf = w[fi];
        if (cnn_ok(bi, kC * kC * kTaps)) vb = w[bi];
    }
    fwd[e] = __float2bfloat16_rn(vf);
    bwd[e] = __float2bfloat16_rn(vb);
}

// The 32 -> 1 layer in the same image: its fp32 weight w = W[0][cin][dy][dx] split exactly
// into three bf16 parts, w = hi + mid + lo (hi = bf16(w), mid = bf16(w - hi), lo = bf16(w -
// hi - mid): two bf16 parts leave at most 8 significant bits, which the third holds), as
// "output channels" 0, 1, 2 (rows 32q + 8 dx + part) of every lane quarter q, so that all
// epilogue warps can read them; the other rows zero.

__global__ void cnn_prep_last_kernel(const float* __restrict__ w, bf16* __restrict__ img)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;      // (chunk, row, lane of 8)
    if (e >= kWImgChunks * kWRows * 8) return;
    const int c8 = e & 7;
    const int row = (e >> 3) % kWRows;
    const int chunk = e / (8 * kWRows);
    if (chunk >= kWChunks) {                                  // no bias step: its bias is added later
        img[e] = __float2bfloat16_rn(0.0f);
        return;
    }
    const int dy = chunk / kPlanes, cin = (chunk % kPlanes) * 8 + c8;
    const int q = row / 32, dx = (row % 32) / 8, part = row % 8;
    float v = 0.0f;
    (void)q;
    if (dx < 3 && part < 3 && cnn_ok((cin * 3 + dy) * 3 + dx, kC * kTaps))
        v = bf16_part(w[(cin * 3 + dy) * 3 + dx], part);
    img[e] = __float2bfloat16_rn(v);
}

// ---------------------------------------------------------------- 32 -> 32 on tcgen05
struct ConvArgs {
    const uint4* in;        // records of `images` images
    const bf16* wimg;       // weight image (kWBytes)
    const float* bias;      // [32] (BIAS), or the last layer's one bias (LAST)
    const uint4* mask;      // records (MASK): output channel c kept where mask's c > 0
    uint4* out;             // records (not LAST)
    const float* ximg;      // LAST: the corrector's input images [images][N][N]
    float* yimg;            // LAST: its output y = x + conv(h) [images][N][N]
    int N, images;
};

// LAST: the 32 -> 1 layer and the skip connection, y = x + b + conv(h), from the weight
// image of cnn_prep_last_kernel: every lane quarter holds the same three rows, and epilogue
// warp (q, eg) takes the 16 columns of groups 2(4 eg + q) and 2(4 eg + q) + 1, adds the
// three weight parts and writes y.
template <bool BIAS, bool RELU, bool MASK, bool LAST>
__global__ void __launch_bounds__(kConvThreads, 1)
cnn_conv32_kernel(ConvArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // run buffers must start on 512-byte atoms: align the carve to 1 KB
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char* wsm = smem;
    unsigned char* ones = smem + kWBytes;                                // bias step's B: bf16 ones
    unsigned char* stages = ones + kOnesBytes;
    unsigned char* scratch = stages + (size_t)kStages * kStageBytes;     // 512 bytes per epilogue warp
    uint64_t* bars = reinterpret_cast<uint64_t*>(scratch + kScratchBytes);
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
            mbar_init(tempty + b, 4 * kEpiGroups);
        }
        mbar_init(wbar, 1);
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "n"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (BIAS) {
        for (int i = threadIdx.x; i < kOnesBytes / 16; i += blockDim.x)
            reinterpret_cast<uint4*>(ones)[i] = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the tensor cores
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---- producer: weights once, then the 3 runs of every tile
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
                const long long m0 = kRecGuard + G.W + (long long)kTileOut * tt;
                mbar_expect_tx(full + s, 3 * kRunCopy);
                unsigned char* dst = stages + (size_t)s * kStageBytes;
#pragma unroll 1
                for (int dy = 0; dy < 3; ++dy) {
                    const long long r0 = m0 + (long long)(dy - 1) * G.W - 1;     // run start
                    const uint4* src = a.in + ((long long)img * G.plane + r0) * kPlanes;
                    if (cnn_span_ok(r0, kRunCopy / kRecBytes, G.plane) && cnn_ok(img, a.images))
                        bulk_g2s(dst + dy * kRunBytes + (int)(r0 & 7) * kRecBytes, src, kRunCopy, full + s);
                }
            }
            // copies still in flight land before the CTA exits
            for (long long j = i - kStages; j < i; ++j)
                if (j >= 0) drain_bar(full + (int)(j % kStages), (uint32_t)(j / kStages) & 1u);
            drain_bar(wbar, 0);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer: per tile 6 MMAs (3 runs x 2 channel halves), A the stacked
            // weights of the run's three taps, B the run's 256 records
            if (wait_bar(wbar, 0, abort_flag)) {
                tc_fence_after();
                const uint32_t wbase = smem_u32(wsm);
                const uint32_t sbase = smem_u32(stages);
                long long i = 0;
                int tt = (int)(blockIdx.x % G.T);
                for (long long t = blockIdx.x; t < total; t += gridDim.x, ++i) {
                    const int s = (int)(i % kStages);
                    const int b = (int)(i % kAcc);
                    if (i > 0) {                               // next tile of this CTA
                        tt += gridDim.x;
                        while (tt >= G.T) tt -= G.T;
                    }
                    const long long m0 = kRecGuard + G.W + (long long)kTileOut * tt;
                    if (!wait_bar(full + s, (uint32_t)(i / kStages) & 1u, abort_flag)) break;
                    if (!wait_bar(tempty + b, ((uint32_t)(i / kAcc) & 1u) ^ 1u, abort_flag)) break;
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(b * kNpix);
                    const uint32_t abase = sbase + (uint32_t)(s * kStageBytes);
#pragma unroll
                    for (int dy = 0; dy < 3; ++dy) {
                        const uint32_t ph = (uint32_t)((m0 - 1 + (long long)(dy - 1) * G.W) & 7);
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
                            const uint64_t ad = smem_desc(wbase + (uint32_t)((dy * kPlanes + 2 * kk) * kWRows * 16),
                                                          kWRows * 16, 128);
                            const uint64_t bd = smem_desc_sw64(abase + (uint32_t)(dy * kRunBytes) +
                                                               ph * kRecBytes + 32u * kk);
                            umma(d, ad, bd, (dy | kk) != 0 ? 1u : 0u);
                        }
                    }
                    if (BIAS)                          // + bias (three parts) x ones, every column
                        umma(d, smem_desc(wbase + (uint32_t)(kWChunks * kWRows * 16), kWRows * 16, 128),
                             smem_desc(smem_u32(ones), kNpix * 16, 128), 1u);
                    umma_commit(empty + s);
                    umma_commit(tfull + b);
                }
            }
            umma_commit(drain);                 // everything issued above has completed ...
            drain_bar(drain, 0);                // ... once this phase does
        }
    } else {
        // ---- epilogue: warpgroup eg (warps 2+4eg .. 5+4eg) takes every tile, 32-column
        // chunks [c0, c0 + 2) of it; each warp reads TMEM lane quarter warp % 4
        const int q = warp & 3;
        const int eg = (warp - 2) >> 2;
        const int etid = threadIdx.x - 64;               // 0 .. 128 kEpiGroups - 1
        // zero the records no tile writes: the guard and top pad row, and the tail
        const long long head = kRecGuard + G.W;
        const long long tail0 = kRecGuard + G.W + (long long)kTileOut * G.T;
        const long long tail = G.plane - tail0;
        const long long nz = LAST ? 0 : (long long)a.images * (head + tail) * kPlanes;   // 16-byte chunks
        for (long long z = (long long)blockIdx.x * (128 * kEpiGroups) + etid; z < nz;
             z += (long long)gridDim.x * (128 * kEpiGroups)) {
            const long long rec = z / kPlanes;
            const int part = (int)(z - rec * kPlanes);
            const long long im = rec / (head + tail);
            const long long r = rec - im * (head + tail);
            const long long o = (im * G.plane + (r < head ? r : tail0 + (r - head))) * kPlanes + part;
            if (cnn_ok(o, (long long)a.images * G.plane * kPlanes)) a.out[o] = make_uint4(0u, 0u, 0u, 0u);
        }
        // TMEM lane 32q + 8dx + g holds output channel 8q + g at tap dx (dx = 3: zero rows).
        // With the 16x256b loads lane t of the warp holds, for g = t / 4 and every group of 8
        // columns, columns 2m and 2m + 1 (m = t % 4) of taps 0 and 1 (load P, lanes 32q ..
        // 32q + 15) and of tap 2 (load Q, lanes 32q + 16 ..).  Output pixel k needs tap dx at
        // column k + dx: for the pair (2m, 2m + 1) the columns 2m + 2, 2m + 3 come from the
        // neighbour m + 1, or for m = 3 from lane m = 0's next group.
        const int m = lane & 3;
        const int nb = (lane & ~3) | ((lane + 1) & 3);
        const int c0 = eg * kChunksPerEpi;               // this group's first 32-column chunk
        const float bias = LAST ? __ldg(a.bias) : 0.0f;   // the hidden layers' biases come from the MMAs
        unsigned char* scr = scratch + (size_t)(warp - 2) * 512;    // [32 px][8 ch] bf16
        long long i = 0;
        int img = (int)(blockIdx.x / G.T), tt = (int)(blockIdx.x % G.T);
        for (long long t = blockIdx.x; t < total; t += gridDim.x, ++i) {
            if (i > 0) {                                 // next tile of this CTA
                tt += gridDim.x;
                while (tt >= G.T) { tt -= G.T; ++img; }
            }
            const int b = (int)(i % kAcc);
            const uint32_t j = (uint32_t)(i / kAcc);
            if constexpr (LAST) {
                // the skip input of this lane's pixel, loaded before the accumulator is waited
                // for (its latency then overlaps the tile's matrix products)
                const int r0 = 2 * (4 * eg + q);             // first of this warp's two groups
                const int px = 8 * r0 + (lane & 15);         // output of the tile
                const unsigned rl = (unsigned)(G.W + kTileOut * tt + px);
                const unsigned ry = rl / (unsigned)G.W;
                const int y = (int)ry - 1, x = (int)(rl - ry * (unsigned)G.W) - 1;
                const bool ok = lane < 16 && px < kTileOut && (unsigned)y < (unsigned)a.N &&
                                (unsigned)x < (unsigned)a.N;
                const size_t pix = ok ? ((size_t)img * a.N + y) * a.N + x : 0;
                long long npx = (long long)a.images * a.N * a.N;
#ifdef FBP_BOUNDS_CHECK
                if (g_cnn_image_limit > 0 && g_cnn_image_limit < a.images)
                    npx = (long long)g_cnn_image_limit * a.N * a.N;
#endif
                const float xin = ok && cnn_ok((long long)pix, npx) ? __ldg(a.ximg + pix) : 0.0f;
                if (!wait_bar(tfull + b, j & 1u, abort_flag)) break;
                tc_fence_after();
                const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * kNpix + 8 * r0);
                uint32_t P[12], Q[12];
                tmem_ld16_x2(tl, P);
                tmem_ld16_x2(tl + (16u << 16), Q);
                if (r0 + 2 < kNpix / 8) {
                    tmem_ld16_x1(tl + 16u, P + 8);
                    tmem_ld16_x1(tl + (16u << 16) + 16u, Q + 8);
                } else {
#pragma unroll
                    for (int u = 8; u < 12; ++u) P[u] = Q[u] = 0u;
                }
                tmem_wait_ld();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(tempty + b);
                // taps summed as in the hidden layers; then channels g = 0, 1, 2 (the weight
                // parts, lanes m, m + 4, m + 8) added: lanes 0..3 hold the conv at columns
                // 8r + 2m, 8r + 2m + 1 of the warp's groups r = 0, 1
                float* vs = reinterpret_cast<float*>(scr);     // [16]: the warp's pixels
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const float pr0 = __uint_as_float(P[4 * r + 2]) + __uint_as_float(Q[4 * r + 1]);
                    const float pr1 = __uint_as_float(P[4 * r + 6]) + __uint_as_float(Q[4 * r + 5]);
                    const uint32_t sa = m == 0 ? Q[4 * r + 4] : Q[4 * r];
                    const float sb = m == 0 ? pr1 : pr0;
                    const float xa = __uint_as_float(__shfl_sync(0xffffffffu, sa, nb));
                    const float xb = __shfl_sync(0xffffffffu, sb, nb);
                    float o0 = (__uint_as_float(P[4 * r]) + __uint_as_float(P[4 * r + 3])) + xa;
                    float o1 = __uint_as_float(P[4 * r + 1]) + xb;
                    o0 = (o0 + __shfl_down_sync(0xffffffffu, o0, 4)) + __shfl_down_sync(0xffffffffu, o0, 8);
                    o1 = (o1 + __shfl_down_sync(0xffffffffu, o1, 4)) + __shfl_down_sync(0xffffffffu, o1, 8);
                    if (lane < 4) {
                        vs[8 * r + 2 * m] = o0;
                        vs[8 * r + 2 * m + 1] = o1;
                    }
                }
                __syncwarp();
                if (ok && cnn_ok((long long)pix, npx)) a.yimg[pix] = xin + (vs[lane] + bias);
                __syncwarp();
                continue;
            }
            if (!wait_bar(tfull + b, j & 1u, abort_flag)) break;
            tc_fence_after();
            const uint32_t tb = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * kNpix);
            // groups 4c0 .. 4c0 + 7 and the first group after them (none after the last chunk)
            constexpr int R = 8;
            uint32_t P[4 * R + 4], Q[4 * R + 4];
            tmem_ld16_x8(tb + (uint32_t)(32 * c0), P);
            tmem_ld16_x8(tb + (16u << 16) + (uint32_t)(32 * c0), Q);
            if (c0 + kChunksPerEpi < kNpix / 32) {
                tmem_ld16_x1(tb + (uint32_t)(32 * (c0 + kChunksPerEpi)), P + 4 * R);
                tmem_ld16_x1(tb + (16u << 16) + (uint32_t)(32 * (c0 + kChunksPerEpi)), Q + 4 * R);
            } else {
#pragma unroll
                for (int u = 4 * R; u < 4 * R + 4; ++u) P[u] = Q[u] = 0u;
            }
            tmem_wait_ld();
            // the accumulator is in registers: hand it back to the MMAs
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty + b);
            // in group r this lane holds tap 0 at columns 2m, 2m + 1 (P[4r], P[4r + 1]), tap 1
            // (P[4r + 2], P[4r + 3]) and tap 2 (Q[4r], Q[4r + 1]).  Outputs 2m and 2m + 1:
            //   out(2m)     = (t0(2m) + t1(2m + 1)) + t2(2m + 2)
            //   out(2m + 1) = t0(2m + 1) + (t1(2m + 2) + t2(2m + 3))
            // the terms of columns 2m + 2, 2m + 3 come from the neighbour m + 1, which sends
            // t2 at its column 2(m+1) and its own sum t1(2(m+1)) + t2(2(m+1) + 1).
            float pre[R + 1];
#pragma unroll
            for (int r = 0; r <= R; ++r)
                pre[r] = __uint_as_float(P[4 * r + 2]) + __uint_as_float(Q[4 * r + 1]);
            // padded-raster position (yy, xx) of this lane's pixel of the first chunk: record
            // kRecGuard + yy W + xx
            const unsigned rel = (unsigned)(G.W + kTileOut * tt + 32 * c0 + lane);
            unsigned yy = rel / (unsigned)G.W;
            unsigned xx = rel - yy * (unsigned)G.W;
#pragma unroll
            for (int h = 0; h < kChunksPerEpi; ++h) {
                uint32_t packed[4];
#pragma unroll
                for (int r4 = 0; r4 < 4; ++r4) {
                    const int r = 4 * h + r4;
                    const uint32_t sa = m == 0 ? Q[4 * r + 4] : Q[4 * r];
                    const float sb = m == 0 ? pre[r + 1] : pre[r];
                    const float xa = __uint_as_float(__shfl_sync(0xffffffffu, sa, nb));
                    const float xb = __shfl_sync(0xffffffffu, sb, nb);
                    float o0 = (__uint_as_float(P[4 * r]) + __uint_as_float(P[4 * r + 3])) + xa;
                    float o1 = __uint_as_float(P[4 * r + 1]) + xb;
                    __nv_bfloat162 pk = __floats2bfloat162_rn(o0, o1);
                    // ReLU after rounding: rounding is monotone and keeps 0, so this equals
                    // rounding the rectified value
                    if (RELU) pk = __hmax2(pk, __floats2bfloat162_rn(0.0f, 0.0f));
                    packed[r4] = *reinterpret_cast<const uint32_t*>(&pk);
                }
                // group r is an 8 x 8 matrix [channel g][pixel 8r + j]: stored transposed, the
                // scratch holds [pixel][channel], i.e. the 16-byte chunk q of 32 pixel records
                stmatrix_x4_trans(smem_u32(scr) + 16u * lane, packed[0], packed[1], packed[2], packed[3]);
                __syncwarp();
                const uint4 wv = reinterpret_cast<const uint4*>(scr)[lane];      // pixel 32(c0+h) + lane
                __syncwarp();
                uint32_t w4[4] = {wv.x, wv.y, wv.z, wv.w};
                const int px = 32 * (c0 + h) + lane;                 // output of the tile
                const int y = (int)yy - 1, x = (int)xx - 1;
                const long long mrec = kRecGuard + (long long)yy * G.W + xx;
                xx += 32;
                while (xx >= (unsigned)G.W) { xx -= (unsigned)G.W; ++yy; }
                if (px < kTileOut) {
                    const bool inside = (unsigned)y < (unsigned)a.N && (unsigned)x < (unsigned)a.N;
                    const long long rec = ((long long)img * G.plane + mrec) * kPlanes + chunk_pos(mrec, q);
                    const bool rec_in = cnn_ok(rec, (long long)a.images * G.plane * kPlanes);
                    if (MASK && inside) {
                        const uint4 mr = rec_in ? a.mask[rec] : make_uint4(0u, 0u, 0u, 0u);
                        const uint32_t mw[4] = {mr.x, mr.y, mr.z, mr.w};
#pragma unroll
                        for (int hh = 0; hh < 4; ++hh) {
                            const float2 mf = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&mw[hh]));
                            const uint32_t keep = (mf.x > 0.0f ? 0x0000ffffu : 0u) | (mf.y > 0.0f ? 0xffff0000u : 0u);
                            w4[hh] &= keep;
                        }
                    }
                    if (rec_in)
                        a.out[rec] = inside ? make_uint4(w4[0], w4[1], w4[2], w4[3]) : make_uint4(0u, 0u, 0u, 0u);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(kTmemCols) : "memory");
    }
}

// ---------------------------------------------------------------- 32 -> 32 weight gradient on tcgen05
// gw[o][c][dy][dx] = sum_p gz[p][o] h[p + (dy-1)W + dx - 1][c]
//                  = sum_q h[q + dx - 1][c] gz[q - (dy-1)W][o]      (q = p + (dy-1)W)
// over every record q of the padded raster (gz and h are zero off the image).  As one GEMM
// with the records as K: D[(dx, c)][(dy, o)] = sum_q A[(dx, c)][q] B[(dy, o)][q], both
// operands "MN-major" in the 64-byte-swizzled layout -- the records themselves, 32 channels
// contiguous per record, 8 records per 512-byte atom.  A (M = 128) is one run of h whose
// four 32-row atoms are the same run shifted by one record each (leading-dimension stride 64
// bytes; atom dx = 3 is a tap that does not exist and is discarded); B (N = 96) is three runs
// of gz, for dy = 0, 1, 2 records m0 + W, m0, m0 - W on, placed L bytes apart with
// L / 64 = -W (mod 8) so that every run's rows keep their records' swizzle phase.  A tile is
// 256 records: 16 MMAs (M = 128, N = 96, K = 16) into one fp32 accumulator that collects all
// of a CTA's tiles; at the end the epilogue warps read it (lane quarter = dx, lane = c,
// column = 32 dy + o) and add it into gw.  The bias gradient is cnn_bias_grad_kernel.
// Roles as in cnn_conv32_kernel: warp 0 copies (one 259-record run of h and three 256-record
// runs of gz per tile into a 3-stage ring), warp 1 issues the MMAs, warps 2-5 read out.
constexpr int kWgTile = 256;                              // records (K) per tile
constexpr int kWgARec = kWgTile + 3;                      // A run: records m0 - 1 .. m0 + 257
constexpr int kWgABytes = 272 * kRecBytes;                // A buffer: phase + run, in atoms
constexpr int kWgBBytes = 50 * 1024;                      // B buffer: three runs L apart + phase
constexpr int kWgStageBytes = kWgABytes + kWgBBytes;
constexpr int kWgStages = 3;
constexpr int kWgThreads = 64 + 128;
constexpr int kWgBarriers = 2 * kWgStages + 2;
constexpr size_t kWgSmem = 1024 + (size_t)kWgStages * kWgStageBytes + kWgBarriers * 8 + 16;
constexpr int kWgCols = 128;                              // TMEM columns (96 used)
constexpr uint32_t kWgIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                              ((uint32_t)(96 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

// MN-major 64-byte-swizzled descriptor: lbo = stride between 32-element atoms along M (or
// N), sbo = stride between groups of 8 K rows
__device__ __forceinline__ uint64_t smem_desc_mn64(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | (4ull << 61);
}

__global__ void __launch_bounds__(kWgThreads, 1)
cnn_wgrad_tc_kernel(const uint4* __restrict__ gz, const uint4* __restrict__ h, float* __restrict__ gw,
                    int N, int images)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char* stages = smem;
    uint64_t* bars = reinterpret_cast<uint64_t*>(stages + (size_t)kWgStages * kWgStageBytes);
    uint64_t* full = bars;                  // [kWgStages] runs landed
    uint64_t* empty = bars + kWgStages;     // [kWgStages] runs consumed by the MMAs
    uint64_t* done = empty + kWgStages;     // every MMA of this CTA complete
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const ActGeom G = act_geom(N);
    const int T = (int)(((long long)N * G.W + kWgTile - 1) / kWgTile);
    const long long total = (long long)T * images;
    // B runs L bytes apart: L / 64 = 256 + (-W mod 8)
    const uint32_t L = (uint32_t)(256 + ((8 - G.W % 8) & 7)) * kRecBytes;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kWgStages; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "n"(kWgCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            long long i = 0;
            int img = (int)(blockIdx.x / T), tt = (int)(blockIdx.x % T);
            for (long long t = blockIdx.x; t < total; t += gridDim.x, ++i) {
                const int s = (int)(i % kWgStages);
                if (i > 0) {
                    tt += gridDim.x;
                    while (tt >= T) { tt -= T; ++img; }
                }
                if (!wait_bar(empty + s, ((uint32_t)(i / kWgStages) & 1u) ^ 1u, abort_flag)) break;
                const long long m0 = kRecGuard + G.W + (long long)kWgTile * tt;
                const long long base = (long long)img * G.plane;
                unsigned char* st = stages + (size_t)s * kWgStageBytes;
                mbar_expect_tx(full + s, kWgARec * kRecBytes + 3 * kWgTile * kRecBytes);
                const long long ra = m0 - 1;                         // A run start
                if (cnn_span_ok(ra, kWgARec, G.plane) && cnn_ok(img, images))
                    bulk_g2s(st + (int)(ra & 7) * kRecBytes, h + (base + ra) * kPlanes, kWgARec * kRecBytes, full + s);
                unsigned char* bb = st + kWgABytes + (int)((m0 + G.W) & 7) * kRecBytes;
#pragma unroll 1
                for (int dy = 0; dy < 3; ++dy) {
                    const long long rb = m0 - (long long)(dy - 1) * G.W;
                    if (cnn_span_ok(rb, kWgTile, G.plane) && cnn_ok(img, images))
                        bulk_g2s(bb + (size_t)dy * L, gz + (base + rb) * kPlanes, kWgTile * kRecBytes, full + s);
                }
            }
            for (long long j = i - kWgStages; j < i; ++j)
                if (j >= 0) drain_bar(full + (int)(j % kWgStages), (uint32_t)(j / kWgStages) & 1u);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t sbase = smem_u32(stages);
            long long i = 0;
            int tt = (int)(blockIdx.x % T);
            for (long long t = blockIdx.x; t < total; t += gridDim.x, ++i) {
                const int s = (int)(i % kWgStages);
                if (i > 0) {
                    tt += gridDim.x;
                    while (tt >= T) tt -= T;
                }
                const long long m0 = kRecGuard + G.W + (long long)kWgTile * tt;
                if (!wait_bar(full + s, (uint32_t)(i / kWgStages) & 1u, abort_flag)) break;
                tc_fence_after();
                const uint32_t a0 = sbase + (uint32_t)(s * kWgStageBytes) + (uint32_t)((m0 - 1) & 7) * kRecBytes;
                const uint32_t b0 = sbase + (uint32_t)(s * kWgStageBytes + kWgABytes) +
                                    (uint32_t)((m0 + G.W) & 7) * kRecBytes;
#pragma unroll 4
                for (int k = 0; k < kWgTile / 16; ++k)
                    umma_idesc(tmem, smem_desc_mn64(a0 + 1024u * k, kRecBytes, 512),
                               smem_desc_mn64(b0 + 1024u * k, L, 512), kWgIdesc, (i | k) != 0 ? 1u : 0u);
                umma_commit(empty + s);
            }
            umma_commit(done);
            drain_bar(done, 0);
        }
    } else {
        // read-out: warp q reads TMEM lane quarter q = dx (q = 3: the discarded tap)
        const int q = warp & 3;
        if (q < 3 && blockIdx.x < total && wait_bar(done, 0, abort_flag)) {
            tc_fence_after();
            for (int c0 = 0; c0 < 96; c0 += 32) {
                uint32_t v[32];
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                             "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                             "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                             : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                               "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                               "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]),
                               "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
                               "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
                               "=r"(v[30]), "=r"(v[31])
                             : "r"(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0));
                tmem_wait_ld();
                const int dy = c0 / 32, c = lane;
#pragma unroll
                for (int o = 0; o < 32; ++o) {
                    const long long gi = ((long long)(o * kC + c) * 3 + dy) * 3 + q;
                    if (cnn_ok(gi, kC * kC * kTaps)) atomicAdd(gw + gi, __uint_as_float(v[o]));
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(kWgCols) : "memory");
    }
}

// gb[o] += sum over every record of gz of channel o (zero off the image): one record per
// thread and step, 32 fp32 sums per thread, reduced across the CTA in shared memory.
__global__ void __launch_bounds__(256)
cnn_bias_grad_kernel(const uint4* __restrict__ gz, float* __restrict__ gb, long long records)
{
    __shared__ float red[kC];
    float acc[kC];
#pragma unroll
    for (int c = 0; c < kC; ++c) acc[c] = 0.0f;
    if (threadIdx.x < kC) red[threadIdx.x] = 0.0f;
    __syncthreads();
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < records;
         r += (long long)gridDim.x * blockDim.x) {
        float v[kC];
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) {
            const long long gi = r * kPlanes + chunk_pos(r, p);
            unpack_record(cnn_ok(gi, records * kPlanes) ? gz[gi] : make_uint4(0u, 0u, 0u, 0u), v + 8 * p);
        }
#pragma unroll
        for (int c = 0; c < kC; ++c) acc[c] += v[c];
    }
#pragma unroll
    for (int c = 0; c < kC; ++c) {
        float x = acc[c];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        if ((threadIdx.x & 31) == 0) atomicAdd(&red[c], x);
    }
    __syncthreads();
    if (threadIdx.x < kC) atomicAdd(gb + threadIdx.x, red[threadIdx.x]);
}

// ---------------------------------------------------------------- 1 -> 32 and 32 -> 1
// First layer: h[p][o] = relu(b[o] + sum_tap w[o][tap] x[p + off(tap)]), fp32 math, written
// as records over the whole plane (zero outside the image).  CTA (row segment, row y,
// image); thread = 4 consecutive pixels x0 .. x0+3 of row y, whose 3 x 6 input window it
// loads once (a 16-byte load and two single values per row).  The weights sit in shared
// memory as [tap][o] and reach registers as 16-byte broadcasts; the 32 channels go in four
// passes of 8 (one record chunk each), two channels per packed fp32 FMA (each channel's sum
// is the same chain of fmaf, bias first and taps in order, as one at a time).  The
// segment's records are assembled in shared memory (a thread's 4 records, then 16 bytes of
// padding, so that the 16-byte writes of a warp fall in distinct banks) and leave as whole
// records in consecutive 16-byte stores.  The row's pad records (x = -1, x = N) are written
// by its first and last threads; grid row y = N zeroes the guard, the top and bottom pad
// rows and the tail.
constexpr int kFirstThreads = 128;
constexpr int kFirstPx = 4;                  // pixels per thread
constexpr int kFirstStage = kFirstPx * kPlanes + 1;        // 16-byte words per thread in shared memory
__global__ void __launch_bounds__(kFirstThreads)
cnn_first_kernel(const float* __restrict__ x, const float* __restrict__ w,
                 uint4* __restrict__ h, int N)
{
    __shared__ __align__(16) float ws[kTaps][kC];
    __shared__ float bs[kC];
    __shared__ uint4 stage[kFirstThreads * kFirstStage];
    for (int e = threadIdx.x; e < kC * kTaps; e += blockDim.x) ws[e % kTaps][e / kTaps] = w[e];
    for (int e = threadIdx.x; e < kC; e += blockDim.x) bs[e] = w[kC * kTaps + e];
    const ActGeom G = act_geom(N);
    const int y = blockIdx.y, img = blockIdx.z;
    uint4* dst = h + (long long)img * G.plane * kPlanes;
    const long long dst_n = G.plane * kPlanes;             // this image's record chunks
    const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
    if (y == N) {
        // records outside every image row: [0, kRecGuard + W) and [kRecGuard + (N+1) W, plane)
        const long long head = kRecGuard + G.W;
        const long long tail0 = kRecGuard + (long long)(N + 1) * G.W;
        const long long n = (head + G.plane - tail0) * kPlanes;
        for (long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x; z < n;
             z += (long long)gridDim.x * blockDim.x) {
            const long long r = z / kPlanes;
            const long long o = (r < head ? r : tail0 + (r - head)) * kPlanes + (int)(z - r * kPlanes);
            if (cnn_ok(o, dst_n)) dst[o] = zero4;
        }
        return;
    }
    __syncthreads();
    const int x0 = kFirstPx * (blockIdx.x * kFirstThreads + threadIdx.x);
    const long long rrow = rec_index(G, y, 0);               // record of pixel (y, 0)
    if (x0 == 0)
#pragma unroll
        for (int p = 0; p < kPlanes; ++p)
            if (cnn_ok((rrow - 1) * kPlanes + p, dst_n)) dst[(rrow - 1) * kPlanes + p] = zero4;
    if (x0 + kFirstPx == N)
#pragma unroll
        for (int p = 0; p < kPlanes; ++p)
            if (cnn_ok((rrow + N) * kPlanes + p, dst_n)) dst[(rrow + N) * kPlanes + p] = zero4;
    const bool live = x0 < N;
    uint4* mine = stage + threadIdx.x * kFirstStage;
    // window xv[dy][k] = x(y + dy - 1, x0 + k - 1), k = 0..5, zero outside the image
    const float* xs = x + (size_t)img * N * N;
    float xv[3][kFirstPx + 2];
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
        const int yy = y + dy - 1;
        if (live && (unsigned)yy < (unsigned)N &&
            cnn_span_ok((long long)yy * N + x0 - (x0 > 0 ? 1 : 0), kFirstPx + (x0 > 0) + (x0 + kFirstPx < N),
                        (long long)N * N)) {
            const float* row = xs + (size_t)yy * N;
            const float4 mid = *reinterpret_cast<const float4*>(row + x0);
            xv[dy][0] = x0 > 0 ? row[x0 - 1] : 0.0f;
            xv[dy][1] = mid.x;
            xv[dy][2] = mid.y;
            xv[dy][3] = mid.z;
            xv[dy][4] = mid.w;
            xv[dy][5] = x0 + kFirstPx < N ? row[x0 + kFirstPx] : 0.0f;
        } else {
#pragma unroll
            for (int k = 0; k < kFirstPx + 2; ++k) xv[dy][k] = 0.0f;
        }
    }
#pragma unroll 1
    for (int c = 0; c < kPlanes; ++c) {                       // channels 8c .. 8c + 7
        float2 acc[kFirstPx][4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 b2 = make_float2(bs[8 * c + 2 * k], bs[8 * c + 2 * k + 1]);
#pragma unroll
            for (int u = 0; u < kFirstPx; ++u) acc[u][k] = b2;
        }
#pragma unroll
        for (int tap = 0; tap < kTaps; ++tap) {
            const int dy = tap / 3, dx = tap % 3;
            const float4 wa = *reinterpret_cast<const float4*>(&ws[tap][8 * c]);
            const float4 wb = *reinterpret_cast<const float4*>(&ws[tap][8 * c + 4]);
            const float2 wk[4] = {make_float2(wa.x, wa.y), make_float2(wa.z, wa.w),
                                  make_float2(wb.x, wb.y), make_float2(wb.z, wb.w)};
#pragma unroll
            for (int u = 0; u < kFirstPx; ++u) {
                const float v = xv[dy][u + dx];
                const float2 v2 = make_float2(v, v);
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[u][k] = __ffma2_rn(wk[k], v2, acc[u][k]);
            }
        }
#pragma unroll
        for (int u = 0; u < kFirstPx; ++u) {
            const long long r = rrow + x0 + u;
            uint32_t w4[4];
#pragma unroll
            for (int hh = 0; hh < 4; ++hh) {
                // ReLU after rounding: rounding is monotone and keeps 0
                const __nv_bfloat162 pk = __hmax2(__floats2bfloat162_rn(acc[u][hh].x, acc[u][hh].y),
                                                  __floats2bfloat162_rn(0.0f, 0.0f));
                w4[hh] = *reinterpret_cast<const uint32_t*>(&pk);
            }
            mine[u * kPlanes + chunk_pos(r, c)] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
        }
    }
    __syncthreads();
    // the segment's records, whole, in consecutive 16-byte words
    const int sx0 = kFirstPx * blockIdx.x * kFirstThreads;   // the segment's first pixel
    const int nw = min(N - sx0, kFirstPx * kFirstThreads) * kPlanes;
    uint4* out = dst + (rrow + sx0) * kPlanes;
    for (int e = threadIdx.x; e < nw; e += kFirstThreads)
        if (cnn_ok((rrow + sx0) * kPlanes + e, dst_n))
            out[e] = stage[(e / (kFirstPx * kPlanes)) * kFirstStage + e % (kFirstPx * kPlanes)];
}

// the 32 channels of record r of one image's records
__device__ __forceinline__ void load_pixel32(float (&v)[kC], const uint4* recs, long long r)
{
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) unpack_record(recs[r * kPlanes + chunk_pos(r, p)], v + 8 * p);
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
    const long long ib = (long long)blockIdx.y * G.plane * kPlanes;
    uint4* dst = g + ib + r * kPlanes;
    if (!cnn_span_ok(r * kPlanes, kPlanes, G.plane * kPlanes)) return;
    if ((unsigned)py >= (unsigned)N || (unsigned)px >= (unsigned)N) {
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) dst[p] = make_uint4(0u, 0u, 0u, 0u);
        return;
    }
    const size_t img = (size_t)blockIdx.y * N * N;
    float v[kTaps];
#pragma unroll
    for (int tap = 0; tap < kTaps; ++tap) {
        const int yy = py - (tap / 3 - 1), xx = px - (tap % 3 - 1);
        v[tap] = (yy >= 0 && yy < N && xx >= 0 && xx < N && cnn_ok((long long)yy * N + xx, (long long)N * N))
                     ? gy[img + (size_t)yy * N + xx] : 0.0f;
    }
    float m[kC];
    load_pixel32(m, h5 + ib, r);
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
        dst[chunk_pos(r, p)] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
    }
}

// ---------------------------------------------------------------- weight gradients (fp32)
// gw[o][c][tap] += sum_p gz[p][o] hp[p + off(tap)][c], gb[o] += sum_p gz[p][o], over all pixels
// of all images.  Persistent CTAs accumulate over 8 x 16-pixel tiles in registers and add
// once into the global gradient (float atomics: the last bits depend on the order).
// Weight gradients of the two 1-channel layers.  Each has a wide side (32 channels, records) and a thin
// side (one channel, an fp32 image); gw[ch][tap] (ch the wide side's channel) sums wide x thin
// over the pixels, one of the two taken at the tap's offset.  WIDE_IS_GZ: first layer, wide =
// the pre-activation gradient gz (unshifted), thin = the input image x (shifted); else last
// layer, wide = the layer's input h (shifted), thin = the output gradient gy (unshifted).
// Per 8 x 16-pixel tile both sides are staged as fp32 in shared memory; thread (group, tap,
// cb) owns channels 4cb .. 4cb+3 of one tap over every fourth pixel of the tile (group =
// pixel mod 4), so each pixel costs one 16-byte and one broadcast shared load for 4 FMAs.
constexpr int kWgThinThreads = 4 * kTaps * 8;
template <bool WIDE_IS_GZ>
__global__ void __launch_bounds__(kWgThinThreads)
cnn_wgrad_thin_kernel(const uint4* __restrict__ wide, const float* __restrict__ thin,
                      float* __restrict__ gw, float* __restrict__ gb, int N, int images)
{
    constexpr int WP = WIDE_IS_GZ ? kTileY * kTileX : kHaloY * kHaloX;   // staged wide pixels
    constexpr int TP = WIDE_IS_GZ ? kHaloY * kHaloX : kTileY * kTileX;   // staged thin pixels
    __shared__ __align__(16) float ws[WP][kC];
    __shared__ float ts[TP];
    const ActGeom G = act_geom(N);
    const int tid = threadIdx.x;
    const int cb = tid & 7, tap = (tid >> 3) % kTaps, grp = tid / (8 * kTaps);
    const int dy = tap / 3, dx = tap % 3;
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f}, accb[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    const int tiles_x = N / kTileX, tiles_y = N / kTileY;
    const long long tiles = (long long)tiles_x * tiles_y * images;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int im = (int)(tile / ((long long)tiles_x * tiles_y));
        const int rem = (int)(tile - (long long)im * tiles_x * tiles_y);
        const int y0 = (rem / tiles_x) * kTileY, x0 = (rem % tiles_x) * kTileX;
        const uint4* wi = wide + (long long)im * G.plane * kPlanes;
        const float* ti = thin + (size_t)im * N * N;
        __syncthreads();                               // previous tile consumed
        for (int e = tid; e < WP * kPlanes; e += kWgThinThreads) {
            const int pix = e / kPlanes, ch = e - pix * kPlanes;
            const long long r = WIDE_IS_GZ ? rec_index(G, y0 + pix / kTileX, x0 + pix % kTileX)
                                           : rec_index(G, y0 - 1 + pix / kHaloX, x0 - 1 + pix % kHaloX);
            float v[8];
            const long long wix = r * kPlanes + chunk_pos(r, ch);
            unpack_record(cnn_ok(wix, G.plane * kPlanes) ? wi[wix] : make_uint4(0u, 0u, 0u, 0u), v);
            *reinterpret_cast<float4*>(&ws[pix][8 * ch]) = make_float4(v[0], v[1], v[2], v[3]);
            *reinterpret_cast<float4*>(&ws[pix][8 * ch + 4]) = make_float4(v[4], v[5], v[6], v[7]);
        }
        for (int e = tid; e < TP; e += kWgThinThreads) {
            float v;
            if (WIDE_IS_GZ) {
                const int gy = y0 - 1 + e / kHaloX, gx = x0 - 1 + e % kHaloX;
                v = (gy >= 0 && gy < N && gx >= 0 && gx < N && cnn_ok((long long)gy * N + gx, (long long)N * N))
                        ? ti[(size_t)gy * N + gx] : 0.0f;
            } else {
                const long long ti_i = (long long)(y0 + e / kTileX) * N + x0 + e % kTileX;
                v = cnn_ok(ti_i, (long long)N * N) ? ti[ti_i] : 0.0f;
            }
            ts[e] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int p = grp; p < kTileY * kTileX; p += 4) {
            const int py = p / kTileX, px = p % kTileX;
            const int ph = (py + dy) * kHaloX + px + dx;               // the tap's halo pixel
            const float4 w4 = *reinterpret_cast<const float4*>(&ws[WIDE_IS_GZ ? p : ph][4 * cb]);
            const float t = ts[WIDE_IS_GZ ? ph : p];
            acc[0] = fmaf(w4.x, t, acc[0]);
            acc[1] = fmaf(w4.y, t, acc[1]);
            acc[2] = fmaf(w4.z, t, acc[2]);
            acc[3] = fmaf(w4.w, t, acc[3]);
            if (WIDE_IS_GZ && tap == 0) {                              // gb[o] = sum gz
                accb[0] += w4.x; accb[1] += w4.y; accb[2] += w4.z; accb[3] += w4.w;
            }
            if (!WIDE_IS_GZ && tap == 0 && cb == 0) accb[0] += t;      // gb[0] = sum gy
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) atomicAdd(gw + (size_t)(4 * cb + k) * kTaps + tap, acc[k]);
    if (WIDE_IS_GZ && tap == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) atomicAdd(gb + 4 * cb + k, accb[k]);
    if (!WIDE_IS_GZ && tap == 0 && cb == 0) atomicAdd(gb, accb[0]);
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

// workspace: the weight images (4 layers x forward and transposed, and the last layer's),
// then `nbuf` record buffers (5 activations and 2 gradients when training, a ping-pong pair
// otherwise)
size_t workspace_bytes(int N, int batch, int train)
{
    const size_t wbytes = (size_t)(4 * 2 + 1) * kWBytes;
    const int nbuf = train ? 5 + 2 : 2;
    return wbytes + (size_t)nbuf * act_bytes(N, batch);
}

struct Ws {
    bf16* wf[4];
    bf16* wb[4];
    bf16* wl;
    uint4* act[7];
};

Ws carve(void* ws, int N, int batch, int train)
{
    Ws w{};
    unsigned char* p = static_cast<unsigned char*>(ws);
    for (int k = 0; k < 4; ++k) { w.wf[k] = reinterpret_cast<bf16*>(p); p += kWBytes; }
    for (int k = 0; k < 4; ++k) { w.wb[k] = reinterpret_cast<bf16*>(p); p += kWBytes; }
    w.wl = reinterpret_cast<bf16*>(p);
    p += kWBytes;
    const size_t a = act_bytes(N, batch);
    for (int k = 0; k < (train ? 7 : 2); ++k) { w.act[k] = reinterpret_cast<uint4*>(p); p += a; }
    return w;
}

constexpr int kMaxCnnDevices = 64;

template <bool BIAS, bool RELU, bool MASK, bool LAST = false>
cudaError_t launch_conv32(const uint4* in, const bf16* wt, const float* bias, const uint4* mask,
                          uint4* out, int N, int batch, int sms, cudaStream_t st,
                          const float* ximg = nullptr, float* yimg = nullptr)
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
            e = cudaFuncSetAttribute(cnn_conv32_kernel<BIAS, RELU, MASK, LAST>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kConvSmem);
            if (e != cudaSuccess) return e;
            done[dev] = true;
        }
    }
    const long long tiles = (long long)act_geom(N).T * batch;
    const int grid = (int)(tiles < sms ? tiles : sms);
    ConvArgs a{in, wt, bias, mask, out, ximg, yimg, N, batch};
    cnn_conv32_kernel<BIAS, RELU, MASK, LAST><<<grid, kConvThreads, kConvSmem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_wgrad_tc(const uint4* gz, const uint4* h, float* gw, float* gb, int N, int batch,
                            int sms, cudaStream_t st)
{
    static std::mutex lock;
    static bool done[kMaxCnnDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxCnnDevices) return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> g(lock);
        if (!done[dev]) {
            e = cudaFuncSetAttribute(cnn_wgrad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kWgSmem);
            if (e != cudaSuccess) return e;
            done[dev] = true;
        }
    }
    const ActGeom G = act_geom(N);
    const long long tiles = ((long long)N * G.W + kWgTile - 1) / kWgTile * batch;
    const int grid = (int)(tiles < sms ? tiles : sms);
    cnn_wgrad_tc_kernel<<<grid, kWgThreads, kWgSmem, st>>>(gz, h, gw, N, batch);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cnn_bias_grad_kernel<<<8 * sms, 256, 0, st>>>(gz, gb, (long long)batch * G.plane);
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
        cnn_prep_weights_kernel<<<(kWImgChunks * kWRows * 8 + 255) / 256, 256, 0, st>>>(
            params + param_offset(k + 1), w.wf[k], w.wb[k]);
    // the first layer: row segments x (N image rows + one row of pad / guard / tail zeroing)
    const dim3 fg((unsigned)((N + kFirstPx * kFirstThreads - 1) / (kFirstPx * kFirstThreads)), N + 1, batch);
    // h1 .. h5 in act[0..4] when saving for the backward pass, else ping-pong in act[0..1]
    auto hbuf = [&](int k) { return save ? w.act[k] : w.act[k & 1]; };
    cnn_first_kernel<<<fg, kFirstThreads, 0, st>>>(x, params, hbuf(0), N);
    const int sms = device_sms();
    if (sms <= 0) return cudaErrorInvalidDevice;
    for (int k = 1; k <= 4; ++k) {
        const float* b = params + param_offset(k) + (size_t)kC * kC * kTaps;
        const cudaError_t e = launch_conv32<true, true, false>(hbuf(k - 1), w.wf[k - 1], b,
                                                               nullptr, hbuf(k), N, batch, sms, st);
        if (e != cudaSuccess) return e;
    }
    cnn_prep_last_kernel<<<(kWImgChunks * kWRows * 8 + 255) / 256, 256, 0, st>>>(params + param_offset(5), w.wl);
    return launch_conv32<false, false, false, true>(hbuf(4), w.wl, params + param_offset(5) + kC * kTaps,
                                                    nullptr, nullptr, N, batch, sms, st, x, y);
}

cudaError_t backward(const float* params, const float* x, const float* gy, float* gparams,
                     void* ws, int N, int batch, int sms, cudaStream_t st)
{
    Ws w = carve(ws, N, batch, 1);
    cudaError_t e = cudaMemsetAsync(gparams, 0, param_count() * sizeof(float), st);
    if (e != cudaSuccess) return e;
    const ActGeom G = act_geom(N);
    const dim3 rg((unsigned)((G.plane + 255) / 256), batch);
    const int wgrid = 8 * sms;             // persistent reductions: enough CTAs to hide their loads
    uint4* g[2] = {w.act[5], w.act[6]};
    // layer 6 (32 -> 1): weights from h5 and gy; gradient into z5
    float* gw = gparams + param_offset(5);
    cnn_wgrad_thin_kernel<false><<<wgrid, kWgThinThreads, 0, st>>>(w.act[4], gy, gw, gw + kC * kTaps, N, batch);
    cnn_last_backward_kernel<<<rg, 256, 0, st>>>(gy, w.act[4], params + param_offset(5), g[0], N);
    int cur = 0;
    // layers 5 .. 2 (32 -> 32): weights from h_{k-1} and g_z_k; gradient into z_{k-1}
    for (int k = 4; k >= 1; --k) {
        gw = gparams + param_offset(k);
        e = launch_wgrad_tc(g[cur], w.act[k - 1], gw, gw + kC * kC * kTaps, N, batch, sms, st);
        if (e != cudaSuccess) return e;
        e = launch_conv32<false, false, true>(g[cur], w.wb[k - 1], nullptr, w.act[k - 1],
                                              g[cur ^ 1], N, batch, sms, st);
        if (e != cudaSuccess) return e;
        cur ^= 1;
    }
    // layer 1 (1 -> 32): weights from x and g_z1
    gw = gparams;
    cnn_wgrad_thin_kernel<true><<<wgrid, kWgThinThreads, 0, st>>>(g[cur], x, gw, gw + kC * kTaps, N, batch);
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

#ifdef FBP_BOUNDS_CHECK
#include "../../include/fbp_check.h"

fbp_status fbp_check_cnn_image_limit(int images)
{
    if (images < 0) return FBP_ERR_INVALID_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return FBP_ERR_CUDA;
    return cudaMemcpyToSymbol(fbp::g_cnn_image_limit, &images, sizeof(int)) == cudaSuccess ? FBP_OK
                                                                                           : FBP_ERR_CUDA;
}
#endif

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
