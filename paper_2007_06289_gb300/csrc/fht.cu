// Linogram resampling (paper Sec. 4.1-4.2, Eq. 14-15) and fast Hough transform back
// projection (Sec. 4.4-4.5, Eq. 16-22).
//
// Hough transform of one quarter (N = 2^n rows i, columns c):
//     H[tau][u] = sum_i L[i][u + d_tau(i)],   tau, u in [0, N),
// with d_tau the dyadic pattern.  The stage recursion
//     H_k[b][tau][u] = H_{k-1}[2b][tau/2][u] + H_{k-1}[2b+1][tau/2][u + ceil(tau/2)]
// is stored "slope bit-reversed": after stage k, strip b's slope tau sits in row
// b*2^k + rev_k(tau).  Stage k is then an in-place butterfly between rows r and r + 2^(k-1)
// (bit k-1 of r clear) with column shifts t and t+1, t = rev_{k-1}(r mod 2^(k-1)):
//     out[r][u]           = in[r][u] + in[r + 2^(k-1)][u + t]
//     out[r + 2^(k-1)][u] = in[r][u] + in[r + 2^(k-1)][u + t + 1]
// Two consecutive stages act on quads of rows {a, a+h, a+2h, a+3h} (h = 2^(k-1), bits k-1
// and k of a clear) with shifts t, t+1 and 2t, 2t+1, 2t+2, so they are done in registers
// ("radix-4 rounds"): one shared-memory read and one write per element per two stages.
// Quads touch disjoint rows, so a round runs in place: each quad belongs to one warp, which
// sweeps its columns left to right in 128-column chunks (a chunk only reads columns that
// later chunks write).
//
// Splitting n = n1 + n2, i = i_hi 2^n1 + i_lo, tau = tau_hi 2^n2 + tau_lo, the pattern
// separates as d_tau(i) = d_{tau_hi}(i_lo) + tau_hi i_hi + d_{tau_lo}(i_hi), so the
// transform runs in two passes, each a small transform in shared memory:
//   pass 1: every block of 2^n1 consecutive rows -> G[i_hi][tau_hi][v] (each row stored
//           shifted by 0..3 columns so that pass 2 starts its reads on 16-byte words)
//   pass 2: for each tau_hi, the 2^n2 rows G[.][tau_hi] sheared by tau_hi * i_hi columns
// (the shear is just a per-row load offset).  Every partial sum is the same float32 sum
// as in the stage recursion, so the result is reproducible bit for bit.
//
// Only outputs u < N are needed; they read linogram row i at columns c <= N-1+i and
// G[i_hi][tau_hi] at columns v < N + (tau_hi+1) i_hi.  Loads beyond these bounds read 0,
// and tiles entirely beyond them are skipped: neither changes a needed output.
#include <type_traits>

#include "fbp_internal.h"

namespace fbp {
namespace {

constexpr int kWB1 = 384;      // pass-1 tile width including the halo of 2^n1 columns
constexpr int kNT1 = 512;      // pass-1 threads
constexpr int kNT2 = 256;      // pass-2 threads
constexpr int kWB2 = 256;      // pass-2 row width: tile plus halo
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int rev_bits(int v, int bits)
{
    return bits == 0 ? 0 : (int)(__brev((unsigned)v) >> (32 - bits));
}

// Asynchronous 4-byte global -> shared copy; an invalid source writes 0.
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src),
                 "r"(valid ? 4 : 0)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// ------------------------------------------------------------------------ resampling
// Detector position in fixed point -> integer bin j (the high word) and fraction f in
// [0, 1] (the low word, rounded to float; f = 1 stands for a position within 2^-25 of j+1).
static_assert(kFixBits == 32, "bin and fraction are the two words of the position");
__device__ __forceinline__ void split_fixed(long long m, int& j, float& f)
{
    j = (int)(m >> 32);
    f = __uint2float_rn((unsigned)m) * 0x1p-32f;
}

// Detector sample j of a row, zero outside [0, M); the load itself is never predicated
// (clamped index), so a batch of them can be in flight together.
__device__ __forceinline__ float ld_bin(const float* __restrict__ row, int M, int j)
{
    const int jc = min(max(j, 0), M - 1);
    const float v = __ldg(row + jc);
    return (unsigned)j < (unsigned)M ? v : 0.0f;
}

__device__ __forceinline__ float ld_bin(const float* __restrict__ row, int M, int j, const Span& sp)
{
    const int jc = min(max(j, 0), M - 1);
    const float v = ldg_in(sp, row + jc);
    return (unsigned)j < (unsigned)M ? v : 0.0f;
}

__device__ __forceinline__ float row_lerp(const float* __restrict__ row, int M, int j, float f)
{
    const float v0 = ld_bin(row, M, j);
    const float v1 = ld_bin(row, M, j + 1);
    return fmaf(f, v1 - v0, v0);
}

// One linogram sample at fixed-point detector position m: w * bilinear(p~, k0 + ft, m),
// with the weight folded into the angle interpolation.
__device__ __forceinline__ float linogram_sample(const RowGeom& g, const float* __restrict__ pt,
                                                 int M, long long m)
{
    int j;
    float f;
    split_fixed(m, j, f);
    const float* rowa = pt + (size_t)g.k0 * M;
    const float va = row_lerp(rowa, M, j, f);
    float vb;
    if (!g.wrap) {
        vb = row_lerp(rowa + M, M, j, f);
    } else {
        // p(pi + theta, r) = p(theta, -r): row 0 with the detector mirrored, m' = (M-1) - m
        int jm;
        float fm;
        split_fixed(((long long)(M - 1) << kFixBits) - m, jm, fm);
        vb = row_lerp(pt, M, jm, fm);
    }
    return fmaf(g.w1, vb, g.w0 * va);
}

// Plain resampling into the stored linogram [count][4][N][2N] (every entry written; a
// geometry row that fails validation resamples to zeros and sets the status word).
__global__ void __launch_bounds__(256)
resample_kernel(const float* __restrict__ filt, float* __restrict__ lin,
                const RowGeom* __restrict__ geom, int N, int K, int M, int count, int* status)
{
    const int W = 2 * N;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int qi = blockIdx.y;                         // q * N + i
    const int s = blockIdx.z;
    if (c >= W) return;
    const RowGeom g = geom[qi];
    const size_t o = ((size_t)s * 4 * N + qi) * W + c;
    if (!in_bounds(status, (long long)o, (long long)count * 4 * N * W)) return;
    if (!row_geom_valid(g, K)) {
        if (c == 0) flag_status(status, (int)FBP_ERR_INTERNAL);
        lin[o] = 0.0f;
        return;
    }
    const float* pt = filt + (size_t)s * K * M;
    lin[o] = linogram_sample(g, pt, M, g.b_fx + g.a_fx * (long long)c);
}

// ------------------------------------------------------------------------ Hough rounds
// Hough rows live in shared memory unpadded, PITCH floats apart with PITCH a multiple of 4,
// so column 4l of any row starts a 16-byte word.  Lane l of a warp owns columns 4l..4l+3 of
// each 128-column chunk and moves them with 16-byte loads and stores: a warp's 16-byte
// accesses cover 512 consecutive bytes, which the shared memory serves without bank
// conflicts.  A shifted read (columns 4l + t + k) loads the aligned words around it and
// picks the values in registers; the pick depends only on t mod 4, which is the same for the
// whole warp, so each of the four cases is compiled separately.
//
// A round hands each thread's results -- four consecutive columns x0..x0+3 of one row,
// the row being the slot-th of the warp's pair or quad -- to a sink.  SmemSink writes them
// back in place (every round but a pass's last); a pass may give its last round a sink that
// stores straight to global memory.  Every lane of the warp calls the sink together.
struct SmemSink {};

__device__ __forceinline__ void ld4(float* v, const float* p)
{
    const float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}

__device__ __forceinline__ void st4(float* p, const float (&o)[4])
{
    *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
}

// Stage 1 (shift 0) on row pairs (2m, 2m+1), in place, one warp per pair.
template <int R, int WB, int PITCH, int NWARPS, class Sink>
__device__ __forceinline__ void round_r2(float* buf, int warp, int lane, const Sink& sink,
                                         int* status)
{
    static_assert(WB % 128 == 0 && PITCH % 4 == 0, "chunked rows");
    for (int pr = warp; pr < R / 2; pr += NWARPS) {
        // furthest float read: row 2pr+1, column (WB - 128) + 4 * 31 + 4
        if (!in_bounds(status, (2 * pr + 1) * PITCH + WB + 0, (long long)R * PITCH)) continue;
        float* A = buf + (2 * pr) * PITCH + 4 * lane;
        float* B = A + PITCH;
        if constexpr (!std::is_same<Sink, SmemSink>::value) {
            sink.begin(0, 2 * pr);
            sink.begin(1, 2 * pr + 1);
        }
#pragma unroll
        for (int xb = 0; xb < WB; xb += 128) {
            float a[4], b[5];
            ld4(a, A + xb);
            ld4(b, B + xb);
            b[4] = B[xb + 4];
            __syncwarp();
            float oa[4], ob[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                oa[k] = a[k] + b[k];
                ob[k] = a[k] + b[k + 1];
            }
            if constexpr (std::is_same<Sink, SmemSink>::value) {
                st4(A + xb, oa);
                st4(B + xb, ob);
            } else {
                sink(0, 2 * pr, xb + 4 * lane, oa);
                sink(1, 2 * pr + 1, xb + 4 * lane, ob);
            }
            __syncwarp();
        }
    }
}

// Stages s and s+1 on the quad {a, a+h, a+2h, a+3h} whose first-stage shift is t = tb + T3
// (tb a multiple of 4).  A..D point at column 4l of the four rows.
template <int T3, int WB, int R, int PITCH, class Sink>
__device__ __forceinline__ void quad_r4(float* A, float* B, float* C, float* D, int tb, int a,
                                        int h, int lane, const Sink& sink, int* status)
{
    // 16-byte words holding rows B, C, D at columns 4l + t + k, 4l + 2t + k, 4l + 3t + k
    constexpr int cb = (2 * T3) & ~3, c3 = (2 * T3) & 3;
    constexpr int db = (3 * T3) & ~3, d3 = (3 * T3) & 3;
    constexpr bool d_three = d3 + 6 > 7;
    // furthest float read: row a + 3h at 3 tb + db + (WB - 128) + 4 * 31 + (d_three ? 11 : 7)
    if (!in_bounds(status, (long long)(a + 3 * h) * PITCH + 3 * tb + db + WB - 4 + (d_three ? 11 : 7),
                   (long long)R * PITCH))
        return;
    const float* Bw = B + tb;
    const float* Cw = C + 2 * tb + cb;
    const float* Dw = D + 3 * tb + db;
    if constexpr (!std::is_same<Sink, SmemSink>::value) {
        sink.begin(0, a);
        sink.begin(1, a + h);
        sink.begin(2, a + 2 * h);
        sink.begin(3, a + 3 * h);
    }
#pragma unroll 1
    for (int xb = 0; xb < WB; xb += 128) {
        float va[4], wb[8], wc[8], wd[12];
        ld4(va, A + xb);
        ld4(wb, Bw + xb);
        ld4(wb + 4, Bw + xb + 4);
        ld4(wc, Cw + xb);
        ld4(wc + 4, Cw + xb + 4);
        ld4(wd, Dw + xb);
        ld4(wd + 4, Dw + xb + 4);
        if constexpr (d_three) ld4(wd + 8, Dw + xb + 8);
        __syncwarp();
        // stage s: rows a, a+h from (A, B) with shifts t, t+1; rows a+2h, a+3h from (C, D)
        // likewise, at the columns stage s+1 will read
        float x0v[4], x1v[4], y0[5], y1[5];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            x0v[k] = va[k] + wb[T3 + k];
            x1v[k] = va[k] + wb[T3 + k + 1];
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            y0[k] = wc[c3 + k] + wd[d3 + k];
            y1[k] = wc[c3 + k + 1] + wd[d3 + k + 2];
        }
        // stage s+1: pairs (a, a+2h) with shift 2t and (a+h, a+3h) with shift 2t+1
        float o0[4], o1[4], o2[4], o3[4];          // rows a, a+h, a+2h, a+3h
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            o0[k] = x0v[k] + y0[k];
            o2[k] = x0v[k] + y0[k + 1];
            o1[k] = x1v[k] + y1[k];
            o3[k] = x1v[k] + y1[k + 1];
        }
        if constexpr (std::is_same<Sink, SmemSink>::value) {
            st4(A + xb, o0);
            st4(B + xb, o1);
            st4(C + xb, o2);
            st4(D + xb, o3);
        } else {
            const int x0 = xb + 4 * lane;
            sink(0, a, x0, o0);
            sink(1, a + h, x0, o1);
            sink(2, a + 2 * h, x0, o2);
            sink(3, a + 3 * h, x0, o3);
        }
        __syncwarp();
    }
}

// Stages s and s+1 (h = 2^(s-1)) on row quads, in place, one warp per quad.
template <int R, int WB, int PITCH, int NWARPS, class Sink>
__device__ __forceinline__ void round_r4(float* buf, int s, int warp, int lane, const Sink& sink,
                                         int* status)
{
    static_assert(WB % 128 == 0 && PITCH % 4 == 0, "chunked rows");
    const int h = 1 << (s - 1);
    for (int qd = warp; qd < R / 4; qd += NWARPS) {
        const int qlo = qd & (h - 1);
        const int a = ((qd >> (s - 1)) << (s + 1)) | qlo;
        const int t = rev_bits(qlo, s - 1);
        float* A = buf + a * PITCH + 4 * lane;
        float* B = A + h * PITCH;
        float* C = A + 2 * h * PITCH;
        float* D = A + 3 * h * PITCH;
        const int tb = t & ~3;
        switch (t & 3) {                                   // the same for the whole warp
            case 0: quad_r4<0, WB, R, PITCH>(A, B, C, D, tb, a, h, lane, sink, status); break;
            case 1: quad_r4<1, WB, R, PITCH>(A, B, C, D, tb, a, h, lane, sink, status); break;
            case 2: quad_r4<2, WB, R, PITCH>(A, B, C, D, tb, a, h, lane, sink, status); break;
            default: quad_r4<3, WB, R, PITCH>(A, B, C, D, tb, a, h, lane, sink, status); break;
        }
    }
}

// All LOGR stages on the R = 2^LOGR rows of `buf`; row j holds slope rev(j).  The last
// round hands its results to `sink` (SmemSink: back into `buf`).
template <int LOGR, int WB, int PITCH, int NWARPS, class Sink>
__device__ __forceinline__ void hough_stages(float* buf, int warp, int lane, const Sink& sink,
                                             int* status)
{
    constexpr int R = 1 << LOGR;
    const SmemSink in_place;
    if constexpr (LOGR == 1) {
        round_r2<R, WB, PITCH, NWARPS>(buf, warp, lane, sink, status);
        __syncthreads();
    } else {
        int s = 1;
        if (LOGR & 1) {
            round_r2<R, WB, PITCH, NWARPS>(buf, warp, lane, in_place, status);
            __syncthreads();
            s = 2;
        }
#pragma unroll 1
        for (; s + 2 < LOGR; s += 2) {
            round_r4<R, WB, PITCH, NWARPS>(buf, s, warp, lane, in_place, status);
            __syncthreads();
        }
        round_r4<R, WB, PITCH, NWARPS>(buf, s, warp, lane, sink, status);
        __syncthreads();
    }
}

// Row pitch: the WB columns, the shifted reads' overhang (at most 3 (R/4 - 1) + 11 columns
// past the last chunk's start word), zero filled; a multiple of 4.
template <int R, int WB>
constexpr int hough_pitch() { return (WB + 3 * (R / 4) + 8 + 3) & ~3; }

// Pass-2 shared floats: the Hough rows of both quarters, the second quarter's rows reused
// for the h quarters' [T2][R+1] transposed result tile.
template <int LOGR2, int T2>
constexpr int pass2_floats()
{
    constexpr int R = 1 << LOGR2;
    constexpr int rows = R * hough_pitch<R, kWB2>();
    return rows + (rows > T2 * (R + 1) ? rows : T2 * (R + 1));
}

// Tile width of a pass (columns it outputs): the WB-column row minus a halo of at least the
// block's slope count, a multiple of 4 so that tiles start on 16-byte words.
template <int R, int WB>
constexpr int tile_width() { return WB - (R > 4 ? R : 4); }

// ------------------------------------------------------------------------ pass 1
// G row layout.  Pass-1 row (block bi, slope tau) holds logical column v at storage index
// v + sh with sh = (-tau bi) mod 4.  The second pass reads that row from v = u0 + tau bi on
// (u0 a multiple of 4), which is then storage u0 + tau bi + sh, a multiple of 4: it copies
// whole 16-byte words.  Only storage [sh, need + sh) is written, need = N + (tau+1) bi.
__device__ __forceinline__ int g_shift(int tau, int bi) { return (-tau * bi) & 3; }

// Last-round sink of pass 1: slot row j holds slope tau = rev(j); its outputs x < T (the
// rest is halo) within the needed region go to G row tau of the block at storage offset
// x + sh from the tile start, sh = g_shift(tau, bi).  The 16-byte word at storage offset x0
// holds x0 - sh .. x0 - sh + 3: the lane's own first 4 - sh values and the last sh of the
// lane before it (for lane 0: lane 31's of the previous 128-column chunk, kept in `carry`),
// moved by warp shuffles.  Partial words at the ends of the region go element by element.
struct GShiftSink {
    float* rows;            // storage offset 0 of G row 0 of this (slice, quarter, block) tile
    int W, T, c0, N, bi, logr, lane;
    Span g;                 // the whole G buffer (checked build: stores outside are dropped)
    mutable float carry[4][3];
    // per slot: the G row, its shift and the end of its stored offsets, set by begin()
    mutable float* dst[4];
    mutable int sh[4], send[4];

    __device__ __forceinline__ void begin(int slot, int j) const
    {
        const int tau = rev_bits(j, logr);
        sh[slot] = g_shift(tau, bi);
        send[slot] = min(T, N + (tau + 1) * bi - c0) + sh[slot];   // storage offsets [sh, send)
        dst[slot] = rows + (size_t)tau * W;
    }

    __device__ __forceinline__ void operator()(int slot, int, int x0, const float (&o)[4]) const
    {
        const int src_lane = (lane + 31) & 31;
        const float r1 = __shfl_sync(kFull, o[1], src_lane);
        const float r2 = __shfl_sync(kFull, o[2], src_lane);
        const float r3 = __shfl_sync(kFull, o[3], src_lane);
        const float p1 = lane == 0 ? carry[slot][0] : r1;
        const float p2 = lane == 0 ? carry[slot][1] : r2;
        const float p3 = lane == 0 ? carry[slot][2] : r3;
        carry[slot][0] = r1;
        carry[slot][1] = r2;
        carry[slot][2] = r3;
        const int lo = sh[slot], hi = send[slot];
        if (x0 >= hi) return;
        float* d = dst[slot] + x0;
        float v[4];
        switch (lo) {                                  // the same for the whole warp
            case 0: v[0] = o[0]; v[1] = o[1]; v[2] = o[2]; v[3] = o[3]; break;
            case 1: v[0] = p3; v[1] = o[0]; v[2] = o[1]; v[3] = o[2]; break;
            case 2: v[0] = p2; v[1] = p3; v[2] = o[0]; v[3] = o[1]; break;
            default: v[0] = p1; v[1] = p2; v[2] = p3; v[3] = o[0]; break;
        }
        if (x0 >= lo && x0 + 4 <= hi) {
            if (g.ok(d) && g.ok(d + 3)) st4(d, v);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (x0 + k >= lo && x0 + k < hi && g.ok(d + k)) d[k] = v[k];
        }
    }
};

struct Pass1Args {
    const float* src;       // filtered sinogram [count][K][pitch] (guarded rows) or
                            // linogram [count][4][N][2N]
    float* g;               // [count][4][N][2N]
    const RowGeom* geom;
    int N, K, M, pitch;
    long long src_n, g_n;   // floats of src and g (checked build)
    int* status;
};

// One warp resamples one linogram row over a WB-column tile: lane l computes columns
// l + 32k at detector positions m0 + k step, angle rows k0 (ra) and k0+1 (ra + pitch) of a
// filtered sinogram whose rows carry kGuard zero bins on each side.  Each batch of kS
// samples issues all of its gathers before combining any of them; the arithmetic is
// linogram_sample's, term for term.  Clamping the bin to [-kGuard, M] keeps bins j and j+1
// inside the guarded row, and a clamped bin only happens when both true bins lie outside
// [0, M), where the guards read 0: the result equals zero padding without any select.
// CLIP zeroes the columns past the trapezoid (column offset 32k > lim).
template <int WB, bool CLIP>
__device__ __forceinline__ void resample_row(float* row, const float* ra, int pitch, int M,
                                             long long m, long long step, float w0, float w1,
                                             int lim, const Span& src)
{
    constexpr int kS = 4;
#pragma unroll
    for (int kb = 0; kb < WB / 32; kb += kS) {
        float l0[kS], l1[kS], l2[kS], l3[kS], fr[kS];
#pragma unroll
        for (int k = 0; k < kS; ++k, m += step) {
            int j;
            split_fixed(m, j, fr[k]);
            const float* pp = ra + min(max(j, -kGuard), M);
            l0[k] = ldg_in(src, pp);
            l1[k] = ldg_in(src, pp + 1);
            l2[k] = ldg_in(src, pp + pitch);
            l3[k] = ldg_in(src, pp + pitch + 1);
        }
#pragma unroll
        for (int k = 0; k < kS; ++k) {
            const float va = fmaf(fr[k], l1[k] - l0[k], l0[k]);
            const float vb = fmaf(fr[k], l3[k] - l2[k], l2[k]);
            const float v = fmaf(w1, vb, w0 * va);
            row[32 * (kb + k)] = (!CLIP || 32 * (kb + k) <= lim) ? v : 0.0f;
        }
    }
}

// Asks L2 for the bins a warp's tile row will gather (angle rows k0 and k0+1 over the
// tile's detector span; nothing for a wrapping row): lanes 0-15 take 32-float lines of row
// k0, lanes 16-31 of row k0+1.  All addresses stay inside the guarded rows.
template <int WB>
__device__ __forceinline__ void prefetch_tile_row(const float* pt, int pitch, int M,
                                                  const RowGeom& gm, int c0, int lane)
{
    if (gm.wrap) return;
    const long long ma = gm.b_fx + gm.a_fx * (long long)c0;
    const long long mb = ma + gm.a_fx * (long long)(WB - 1);
    const int ja = max((int)((ma < mb ? ma : mb) >> kFixBits), -kGuard);
    const int jb = min((int)((ma < mb ? mb : ma) >> kFixBits) + 1, M + kGuard - 1);
    if (ja > jb) return;
    const float* r = pt + (size_t)gm.k0 * pitch + (lane >= 16 ? pitch : 0);
    const float* a = r + min(ja + 32 * (lane & 15), jb);
    asm volatile("prefetch.global.L2 [%0];\n" ::"l"(a));
}

// CTA = (column tile, quarter * blocks + block, slice).  Resamples (or loads) the block's
// 2^LOGR linogram rows over the tile plus halo, runs LOGR stages, writes G.
template <int LOGR, bool FROM_LIN>
__global__ void __launch_bounds__(kNT1, 2)
pass1_kernel(Pass1Args a)
{
    constexpr int R = 1 << LOGR;
    constexpr int WB = kWB1;
    constexpr int T = tile_width<R, WB>();
    constexpr int PITCH = hough_pitch<R, WB>();
    constexpr int NWARPS = kNT1 / 32;
    extern __shared__ __align__(16) float buf[];

    const int N = a.N, W = 2 * N;
    const int nblocks = N >> LOGR;
    const int q = blockIdx.y / nblocks;
    const int bi = blockIdx.y - q * nblocks;
    const int s = blockIdx.z;
    const int c0 = blockIdx.x * T;
    if (c0 >= N + R * bi) return;                      // nothing needed in this tile
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t lin_q = ((size_t)s * 4 + q) * N;      // row index base of this quarter
    const Span src{a.src, a.src_n, a.status};

    if (FROM_LIN) {
        for (int idx = threadIdx.x; idx < R * WB; idx += kNT1) {
            const int j = idx / WB;
            const int x = idx - j * WB;
            const int i = bi * R + j;
            const int c = c0 + x;
            const float* sp = a.src + (lin_q + i) * W + c;
            const bool ok = c <= N - 1 + i && src.ok(sp);
            cp_async4(buf + j * PITCH + x, ok ? sp : a.src, ok);
        }
    } else {
        // One warp per linogram row, lane = column within each 32-column group.  Rows of
        // the filtered sinogram are `pitch` floats apart with kGuard zero bins on each side;
        // pt points at bin 0 of row 0 of this slice.
        const float* pt = a.src + (size_t)s * a.K * a.pitch + kGuard;
        const int M = a.M;
        const int pitch = a.pitch;
        constexpr int kS = 4;
        // each warp takes RPW consecutive rows, which mostly share their angle rows (L1
        // reuse); start all of them on their way into L2 before gathering any
        constexpr int RPW = R >= NWARPS ? R / NWARPS : 1;
        for (int jj = 0; jj < RPW; ++jj) {
            const int j = warp * RPW + jj;
            if (j >= R) break;
            const int i = bi * R + j;
            const RowGeom gm = a.geom[q * N + i];
            if (c0 <= N - 1 + i && row_geom_valid(gm, a.K))
                prefetch_tile_row<WB>(pt, pitch, M, gm, c0, lane);
        }
        for (int jj = 0; jj < RPW; ++jj) {
            const int j = warp * RPW + jj;
            if (j >= R) break;
            const int i = bi * R + j;
            const int limit = N - 1 + i;
            float* row = buf + j * PITCH + lane;
            if (c0 > limit) {                                  // tile past the trapezoid
#pragma unroll
                for (int k = 0; k < WB / 32; ++k) row[32 * k] = 0.0f;
                continue;
            }
            const RowGeom gm = a.geom[q * N + i];
            if (!row_geom_valid(gm, a.K)) {                   // rejected row: zeros
                if (lane == 0 && blockIdx.x == 0) flag_status(a.status, (int)FBP_ERR_INTERNAL);
#pragma unroll
                for (int k = 0; k < WB / 32; ++k) row[32 * k] = 0.0f;
                continue;
            }
            const float* ra = pt + (size_t)gm.k0 * pitch;
            const long long m0 = gm.b_fx + gm.a_fx * (long long)(c0 + lane);
            const long long step = gm.a_fx * 32;
            if (!gm.wrap) {
                if (c0 + WB - 1 <= limit)                      // whole tile inside the trapezoid
                    resample_row<WB, false>(row, ra, pitch, M, m0, step, gm.w0, gm.w1, 0, src);
                else
                    resample_row<WB, true>(row, ra, pitch, M, m0, step, gm.w0, gm.w1,
                                           limit - c0 - lane, src);
                continue;
            }
            const float* rb = pt;                              // wrap: row 0, mirrored
            const long long mirror = ((long long)(M - 1) << kFixBits);
#pragma unroll
            for (int kb = 0; kb < WB / 32; kb += kS) {
                float a0[kS], a1[kS], b0[kS], b1[kS], fa[kS], fb[kS];
#pragma unroll
                for (int k = 0; k < kS; ++k) {
                    const long long m = m0 + step * (kb + k);
                    int ja, jb;
                    split_fixed(m, ja, fa[k]);
                    if (gm.wrap) split_fixed(mirror - m, jb, fb[k]);
                    else { jb = ja; fb[k] = fa[k]; }
                    a0[k] = ld_bin(ra, M, ja, src);
                    a1[k] = ld_bin(ra, M, ja + 1, src);
                    b0[k] = ld_bin(rb, M, jb, src);
                    b1[k] = ld_bin(rb, M, jb + 1, src);
                }
#pragma unroll
                for (int k = 0; k < kS; ++k) {
                    const float va = fmaf(fa[k], a1[k] - a0[k], a0[k]);
                    const float vb = fmaf(fb[k], b1[k] - b0[k], b0[k]);
                    const float v = fmaf(gm.w1, vb, gm.w0 * va);
                    row[32 * (kb + k)] = (c0 + lane + 32 * (kb + k) <= limit) ? v : 0.0f;
                }
            }
        }
    }
    for (int j = warp; j < R; j += NWARPS)
        for (int p = WB + lane; p < PITCH; p += 32) buf[j * PITCH + p] = 0.0f;
    if (FROM_LIN) cp_async_wait_all();
    __syncthreads();

    const GShiftSink out{a.g + (lin_q + (size_t)bi * R) * W + c0, W, T, c0, N, bi, LOGR, lane,
                         Span{a.g, a.g_n, a.status}, {}};
    hough_stages<LOGR, WB, PITCH, NWARPS>(buf, warp, lane, out, a.status);
}

// ------------------------------------------------------------------------ pass 2
struct Pass2Args {
    const float* g;         // [count][4][N][2N]
    float* img;             // [count][N][N]
    float* const* img_tab;  // optional: slice s's image at img_tab[s]
    int N, n1;
    long long g_n;          // floats of g (checked build)
    int* status;
};

// 16-byte asynchronous copy; src_bytes = 0 writes zeros (src is then not read).
__device__ __forceinline__ void cp_async16(float* dst, const float* src, int src_bytes)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int N_PENDING>
__device__ __forceinline__ void cp_async_wait_group()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N_PENDING) : "memory");
}

// Whole G rows of the second pass arrive by 1-D bulk copies counted on an mbarrier: every
// issuing lane adds its bytes to the barrier's transaction count before its copy, and one
// thread arrives once all have (after a CTA barrier), so the phase completes when the last
// copy has landed.
__device__ __forceinline__ unsigned smem_addr(const void* p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void bar_init(uint64_t* bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void bar_expect(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes) : "memory");
}

__device__ __forceinline__ void bar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void bulk_row(float* dst, const float* src, unsigned bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}

// Waits for phase 0 of `bar`, for at most about a second (then sets FBP_ERR_TIMEOUT in the
// status word and returns: the copies are lost, nothing hangs).
__device__ __forceinline__ void bar_wait(uint64_t* bar, int* status)
{
    unsigned long long t0 = 0;
    for (unsigned it = 0;; ++it) {
        unsigned ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
                     " selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(ok) : "r"(smem_addr(bar)) : "memory");
        if (ok) return;
        unsigned long long now;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
        if (it == 0) t0 = now;
        else if (now - t0 > 1000000000ull) {
            flag_status(status, (int)FBP_ERR_TIMEOUT);
            return;
        }
    }
}

// CTA = (tile of T2 intercepts u, slope group tau_hi, slice).  Runs the second pass for the
// '-' quarter on u in [x0, x0+T2) and for the '+' quarter on the mirrored range, adds them
// (F_- + F_+), and either stores the sum into the image (v quarters: [y = tau][x = u]) or
// adds it to the image through a shared-memory transpose (h quarters: [y = u][x = tau]).
// Launched for the v quarters first and the h quarters second, so each pixel ends as
// (F_v- + F_v+) + (F_h- + F_h+).  Each h CTA asks L2 for its image rows when it starts, so
// that the read-modify-write at its end finds them there, and the h launch takes the slices
// in reverse order, starting on the images the v launch wrote last.  Both quarters' rows
// are requested up front (one bulk copy per row that lies wholly inside its stored range,
// counted on the quarter's mbarrier; 16-byte asynchronous copies with zero fill for the
// rows at the ends of the range), so the second quarter's copies run behind the first
// quarter's stages.
template <int LOGR2, int T2, bool HORIZ>
__global__ void __launch_bounds__(kNT2, 3)
pass2_kernel(Pass2Args a)
{
    constexpr int R = 1 << LOGR2;
    constexpr int WB = kWB2;                   // two 128-column chunks: tile plus halo
    static_assert(T2 + R <= WB && T2 % 4 == 0, "pass-2 tile");
    constexpr int PITCH = hough_pitch<R, WB>();
    constexpr int NWARPS = kNT2 / 32;
    constexpr int TP = R + 1;                  // [T2][R + 1] transposed tile (h quarters)
    extern __shared__ __align__(16) float buf[];
    float* const hb0 = buf;                    // '-' quarter rows
    float* const hb1 = buf + R * PITCH;        // '+' quarter rows, later the transposed tile

    const int N = a.N, W = 2 * N;
    const int R1 = 1 << a.n1;
    const int x0 = blockIdx.x * T2;            // the last tile may run past N
    const int nx = min(T2, N - x0);            // intercepts of this tile inside the image
    const int tau_hi = blockIdx.y;
    const int s = HORIZ ? (int)gridDim.z - 1 - (int)blockIdx.z : (int)blockIdx.z;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* img = a.img_tab ? a.img_tab[s] : a.img + (size_t)s * N * N;
    const Span gs{a.g, a.g_n, a.status};
    const Span is{img, (long long)N * N, a.status};    // this slice's image
    if constexpr (HORIZ) {
        // image row x0 + t from column tau_hi R on: the first 128-byte line of its R columns
        // (all of them while R <= 32)
        const float* ir = img + (size_t)(x0 + (int)threadIdx.x) * N + tau_hi * R;
        if ((int)threadIdx.x < nx && is.ok(ir)) asm volatile("prefetch.global.L2 [%0];" ::"l"(ir));
    }
    __shared__ uint64_t rows_landed[2];                // per quarter: its bulk row copies
    if (threadIdx.x == 0) {
        bar_init(&rows_landed[0]);
        bar_init(&rows_landed[1]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
        const int q = (HORIZ ? 2 : 0) + half;
        // '-' quarter: u = x0 + xx; '+' quarter: u = N-1-(x0+xx), i.e. column T2-1-xx of a
        // tile starting at N - x0 - T2 (negative for a partial last tile: those columns
        // only feed intercepts outside the image)
        const int uo = half == 0 ? x0 : N - x0 - T2;
        const float* gq = a.g + ((size_t)s * 4 + q) * N * W;
        float* hb = half == 0 ? hb0 : hb1;
        for (int ih = warp; ih < R; ih += NWARPS) {
            // row (ih, tau_hi) from logical column uo + tau_hi ih on: storage sb + x, with the
            // stored columns [sh, need + sh)
            const int sh = g_shift(tau_hi, ih);
            const int lo = sh;
            const int hi = N + (tau_hi + 1) * ih + sh;
            const int sb = uo + tau_hi * ih + sh;
            const float* grow = gq + ((size_t)ih * R1 + tau_hi) * W;
            float* drow = hb + ih * PITCH;
            if (sb >= lo && sb + WB <= hi && gs.ok(grow + sb) && gs.ok(grow + sb + WB - 1)) {
                if (lane == 0) {
                    bar_expect(&rows_landed[half], WB * 4);
                    bulk_row(drow, grow + sb, WB * 4, &rows_landed[half]);
                }
                for (int p = WB + lane; p < PITCH; p += 32) drow[p] = 0.0f;
                continue;
            }
#pragma unroll
            for (int m = lane; m < WB / 4; m += 32) {
                const int st = sb + 4 * m;
                if (st >= lo && st + 4 <= hi && gs.ok(grow + st) && gs.ok(grow + st + 3)) {
                    cp_async16(drow + 4 * m, grow + st, 16);
                } else if (st + 4 <= lo || st >= hi) {
                    cp_async16(drow + 4 * m, grow, 0);
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const bool ok = st + k >= lo && st + k < hi && gs.ok(grow + st + k);
                        cp_async4(drow + 4 * m + k, ok ? grow + st + k : grow, ok);
                    }
                }
            }
            for (int p = WB + lane; p < PITCH; p += 32) drow[p] = 0.0f;
        }
        cp_async_commit();
    }
    __syncthreads();                                   // every bulk copy is counted
    if (threadIdx.x == 0) {
        bar_arrive(&rows_landed[0]);
        bar_arrive(&rows_landed[1]);
    }
    cp_async_wait_group<1>();
    bar_wait(&rows_landed[0], a.status);
    __syncthreads();
    hough_stages<LOGR2, WB, PITCH, NWARPS>(hb0, warp, lane, SmemSink{}, a.status);
    cp_async_wait_group<0>();
    bar_wait(&rows_landed[1], a.status);
    __syncthreads();
    hough_stages<LOGR2, WB, PITCH, NWARPS>(hb1, warp, lane, SmemSink{}, a.status);

    // F_- + F_+ for slot row j (slope tau_lo = rev(j)) at intercept x0 + xx: columns xx of
    // hb0 and T2-1-xx of hb1, taken as 16-byte words (the second one reversed).
    if constexpr (!HORIZ) {
        for (int j = warp; j < R; j += NWARPS) {
            float* out = img + (size_t)(tau_hi * R + rev_bits(j, LOGR2)) * N + x0;
            const float* r0 = hb0 + j * PITCH;
            const float* r1 = hb1 + j * PITCH;
            for (int xx = 4 * lane; xx < nx; xx += 128) {
                float va[4], vb[4], o[4];
                ld4(va, r0 + xx);
                ld4(vb, r1 + T2 - 4 - xx);
#pragma unroll
                for (int k = 0; k < 4; ++k) o[k] = va[k] + vb[3 - k];
                if (is.ok(out + xx) && is.ok(out + xx + 3)) st4(out + xx, o);
            }
        }
    } else {
        // h quarters: the sums in place into hb0, then transposed into [xx][tau_lo] (in
        // hb1's space), then added to image rows x0 + xx, columns tau_hi R .. + R.
        for (int j = warp; j < R; j += NWARPS) {
            float* r0 = hb0 + j * PITCH;
            const float* r1 = hb1 + j * PITCH;
            for (int xx = 4 * lane; xx < T2; xx += 128) {
                float va[4], vb[4], o[4];
                ld4(va, r0 + xx);
                ld4(vb, r1 + T2 - 4 - xx);
#pragma unroll
                for (int k = 0; k < 4; ++k) o[k] = va[k] + vb[3 - k];
                st4(r0 + xx, o);
            }
        }
        __syncthreads();
        float* tt = hb1;
        for (int tl = warp; tl < R; tl += NWARPS) {
            const float* r0 = hb0 + rev_bits(tl, LOGR2) * PITCH;
            for (int xx = lane; xx < nx; xx += 32) tt[xx * TP + tl] = r0[xx];
        }
        __syncthreads();
        // read-modify-write of the image rows, a batch of kB rows per warp at a time so that
        // the batch's loads are in flight together
        constexpr int kB = 7;
        for (int xb = warp; xb < nx; xb += NWARPS * kB) {
            for (int tl = lane; tl < R; tl += 32) {
                float* out = img + (size_t)(x0 + xb) * N + tau_hi * R + tl;
                const float* src = tt + xb * TP + tl;
                float v[kB];
#pragma unroll
                for (int u = 0; u < kB; ++u)
                    if (xb + NWARPS * u < nx && is.ok(out + (size_t)NWARPS * u * N))
                        v[u] = out[(size_t)NWARPS * u * N];
#pragma unroll
                for (int u = 0; u < kB; ++u)
                    if (xb + NWARPS * u < nx && is.ok(out + (size_t)NWARPS * u * N))
                        out[(size_t)NWARPS * u * N] = v[u] + src[NWARPS * u * TP];
            }
        }
    }
}

// Single-pass sizes (n <= 6): G already holds the quarter images H_q[tau][u]; sum them.
__global__ void __launch_bounds__(256)
combine_kernel(const float* __restrict__ g, float* __restrict__ img, float* const* img_tab, int N,
               long long g_n, int* status)
{
    const int W = 2 * N;
    const int s = blockIdx.y;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N * N) return;
    const int y = p / N;
    const int x = p - y * N;
    const float* h = g + (size_t)s * 4 * N * W;
    const size_t qs = (size_t)N * W;
    const Span gs{g, g_n, status};
    const float v = ldg_in(gs, h + (size_t)y * W + x) + ldg_in(gs, h + qs + (size_t)y * W + (N - 1 - x));
    const float hh = ldg_in(gs, h + 2 * qs + (size_t)x * W + y) + ldg_in(gs, h + 3 * qs + (size_t)x * W + (N - 1 - y));
    (img_tab ? img_tab[s] : img + (size_t)s * N * N)[p] = v + hh;
}

// ------------------------------------------------------------------------ launchers
template <int LOGR>
constexpr size_t pass1_smem() { return (size_t)(1 << LOGR) * hough_pitch<(1 << LOGR), kWB1>() * sizeof(float); }

template <int LOGR2, int T2>
constexpr size_t pass2_smem() { return (size_t)pass2_floats<LOGR2, T2>() * sizeof(float); }

// floats of pass 1's input: a stored linogram, or the guarded filtered sinograms
template <bool FROM_LIN>
long long from_lin_floats(const fbp_plan_s* p, int count)
{
    return FROM_LIN ? (long long)count * (long long)lin_floats(p)
                    : (long long)count * p->K * filt_pitch(p);
}

template <int LOGR, bool FROM_LIN>
cudaError_t launch_pass1_t(const fbp_plan_s* p, const float* src, float* g, int count,
                           cudaStream_t st)
{
    constexpr int R = 1 << LOGR;
    constexpr int T = tile_width<R, kWB1>();
    const int nblocks = p->N >> LOGR;
    const int max_cols = p->N + R * (nblocks - 1);
    dim3 grid((max_cols + T - 1) / T, 4 * nblocks, count);
    const long long src_n = from_lin_floats<FROM_LIN>(p, count);
    Pass1Args a{src, g, p->d_geom, p->N, p->K, p->M, filt_pitch(p), src_n,
                (long long)count * (long long)lin_floats(p), p->d_status};
    pass1_kernel<LOGR, FROM_LIN><<<grid, kNT1, pass1_smem<LOGR>(), st>>>(a);
    return cudaGetLastError();
}

template <int LOGR2, int T2, bool HORIZ>
cudaError_t launch_pass2_t(const fbp_plan_s* p, const float* g, float* img, int count,
                           cudaStream_t st, float* const* img_tab)
{
    dim3 grid((p->N + T2 - 1) / T2, p->N >> LOGR2, count);
    Pass2Args a{g, img, img_tab, p->N, p->n1, (long long)count * (long long)lin_floats(p),
                p->d_status};
    pass2_kernel<LOGR2, T2, HORIZ><<<grid, kNT2, pass2_smem<LOGR2, T2>(), st>>>(a);
    return cudaGetLastError();
}

template <int LOGR, bool FROM_LIN>
cudaError_t set_p1_attr()
{
    return cudaFuncSetAttribute(pass1_kernel<LOGR, FROM_LIN>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pass1_smem<LOGR>());
}

template <int LOGR2, int T2, bool HORIZ>
cudaError_t set_p2_attr()
{
    return cudaFuncSetAttribute(pass2_kernel<LOGR2, T2, HORIZ>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)pass2_smem<LOGR2, T2>());
}

// Second-pass tile: T2 intercepts plus the 2^n2 halo fit the two 128-column chunks.
template <int LOGR2>
constexpr int pass2_tile() { return tile_width<(1 << LOGR2), kWB2>(); }

template <int LOGR2, bool HORIZ>
cudaError_t launch_pass2_n(const fbp_plan_s* p, const float* g, float* img, int count,
                           cudaStream_t st, float* const* img_tab)
{
    return launch_pass2_t<LOGR2, pass2_tile<LOGR2>(), HORIZ>(p, g, img, count, st, img_tab);
}

}  // namespace

cudaError_t prepare_fht_kernels()
{
    cudaError_t e = cudaSuccess;
#define FBP_P1(L)                                              \
    if (e == cudaSuccess) e = set_p1_attr<L, false>();         \
    if (e == cudaSuccess) e = set_p1_attr<L, true>();
    FBP_P1(1) FBP_P1(2) FBP_P1(3) FBP_P1(4) FBP_P1(5) FBP_P1(6)
#undef FBP_P1
#define FBP_P2(L)                                                      \
    if (e == cudaSuccess) e = set_p2_attr<L, pass2_tile<L>(), false>();  \
    if (e == cudaSuccess) e = set_p2_attr<L, pass2_tile<L>(), true>();
    FBP_P2(1) FBP_P2(2) FBP_P2(3) FBP_P2(4) FBP_P2(5) FBP_P2(6)
#undef FBP_P2
    return e;
}

cudaError_t launch_resample(const fbp_plan_s* p, const float* filt, float* lin, int count,
                            cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    dim3 grid((2 * p->N + 255) / 256, 4 * p->N, count);
    resample_kernel<<<grid, 256, 0, st>>>(filt, lin, p->d_geom, p->N, p->K, p->M, count,
                                          p->d_status);
    return cudaGetLastError();
}

cudaError_t launch_pass1(const fbp_plan_s* p, const float* src, bool from_lin, float* g,
                         int count, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    switch (p->n1 * 2 + (from_lin ? 1 : 0)) {
#define FBP_C(L)                                                        \
    case 2 * L: return launch_pass1_t<L, false>(p, src, g, count, st); \
    case 2 * L + 1: return launch_pass1_t<L, true>(p, src, g, count, st);
        FBP_C(1) FBP_C(2) FBP_C(3) FBP_C(4) FBP_C(5) FBP_C(6)
#undef FBP_C
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_pass2(const fbp_plan_s* p, const float* g, float* img, int count,
                         bool horizontal, cudaStream_t st, float* const* img_tab)
{
    if (count <= 0) return cudaSuccess;
    if (p->n2 == 0) {
        if (horizontal) return cudaSuccess;            // the sum kernel does all quarters
        dim3 grid((p->N * p->N + 255) / 256, count);
        combine_kernel<<<grid, 256, 0, st>>>(g, img, img_tab, p->N,
                                             (long long)count * (long long)lin_floats(p), p->d_status);
        return cudaGetLastError();
    }
    switch (p->n2 * 2 + (horizontal ? 1 : 0)) {
#define FBP_C(L)                                                              \
    case 2 * L: return launch_pass2_n<L, false>(p, g, img, count, st, img_tab);       \
    case 2 * L + 1: return launch_pass2_n<L, true>(p, g, img, count, st, img_tab);
        FBP_C(1) FBP_C(2) FBP_C(3) FBP_C(4) FBP_C(5) FBP_C(6)
#undef FBP_C
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fbp
