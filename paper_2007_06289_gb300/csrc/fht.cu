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
// Splitting n = n1 + n2, i = i_hi 2^n1 + i_lo, tau = tau_hi 2^n2 + tau_lo, the pattern
// separates as d_tau(i) = d_{tau_hi}(i_lo) + tau_hi i_hi + d_{tau_lo}(i_hi), so the
// transform runs in two passes, each a small transform in shared memory:
//   pass 1: every block of 2^n1 consecutive rows -> G[i_hi][tau_hi][v]
//   pass 2: for each tau_hi, the 2^n2 rows G[.][tau_hi] sheared by tau_hi * i_hi columns
// (the shear is just a per-row load offset).  Every partial sum is the same float32 sum
// as in the stage recursion, so the result is reproducible bit for bit.
//
// Only outputs u < N are needed; they read linogram row i at columns c <= N-1+i and
// G[i_hi][tau_hi] at columns v < N + (tau_hi+1) i_hi.  Loads beyond these bounds read 0,
// and tiles entirely beyond them are skipped: neither changes a needed output.
#include "fbp_internal.h"

namespace fbp {
namespace {

constexpr int kP1Threads = 256;
constexpr int kP1Tile = 64;      // pass-1 output columns per CTA
constexpr int kP2Threads = 256;
constexpr int kP2Tile = 64;      // pass-2 image tile edge

__device__ __forceinline__ int rev_bits(int v, int bits)
{
    return bits == 0 ? 0 : (int)(__brev((unsigned)v) >> (32 - bits));
}

// Detector position m = A*c + B in double-float, returned as integer part j and
// fraction f in [0, 1).
__device__ __forceinline__ void detector_pos(const RowGeom& g, int c, int& j, float& f)
{
    const float cf = (float)c;
    const float p = g.a_hi * cf;
    const float pe = fmaf(g.a_hi, cf, -p);            // exact rounding error of the product
    const float s = p + g.b_hi;
    const float bb = s - p;
    const float se = (p - (s - bb)) + (g.b_hi - bb);  // exact rounding error of the sum
    const float lo = se + pe + fmaf(g.a_lo, cf, g.b_lo);
    const float fl = floorf(s);
    const float fr = (s - fl) + lo;                   // s - fl is exact
    const float adj = floorf(fr);
    j = (int)fl + (int)adj;
    f = fr - adj;
}

__device__ __forceinline__ float row_lerp(const float* __restrict__ row, int M, int j, float f)
{
    const float v0 = (j >= 0 && j < M) ? __ldg(row + j) : 0.0f;
    const float v1 = (j + 1 >= 0 && j + 1 < M) ? __ldg(row + j + 1) : 0.0f;
    return fmaf(f, v1 - v0, v0);
}

// One linogram sample: w * bilinear(p~, k0 + ft, m(c)).
__device__ __forceinline__ float linogram_sample(const RowGeom& g, const float* __restrict__ pt,
                                                 int K, int M, int c)
{
    int j;
    float f;
    detector_pos(g, c, j, f);
    const float* rowa = pt + (size_t)g.k0 * M;
    const float va = row_lerp(rowa, M, j, f);
    float vb;
    if (!g.wrap) {
        vb = row_lerp(rowa + M, M, j, f);
    } else {
        // p(pi + theta, r) = p(theta, -r): mirrored detector on row 0; m' = (M-1) - m
        int jm;
        float fm;
        if (f == 0.0f) { jm = M - 1 - j; fm = 0.0f; }
        else { jm = M - 2 - j; fm = 1.0f - f; }
        vb = row_lerp(pt, M, jm, fm);
    }
    (void)K;
    return g.w * fmaf(g.ft, vb - va, va);
}

// ---------------------------------------------------------------------------------------
// Plain resampling into the stored linogram [count][4][N][2N] (every entry written).
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
resample_kernel(const float* __restrict__ filt, float* __restrict__ lin,
                const RowGeom* __restrict__ geom, int N, int K, int M)
{
    const int W = 2 * N;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int qi = blockIdx.y;                         // q * N + i
    const int s = blockIdx.z;
    if (c >= W) return;
    const RowGeom g = geom[qi];
    const float* pt = filt + (size_t)s * K * M;
    lin[((size_t)s * 4 * N + qi) * W + c] = linogram_sample(g, pt, K, M, c);
}

// ---------------------------------------------------------------------------------------
// Shared-memory Hough stages on R = 2^LOGR rows of width WB (bit-reversed slope rows).
// Reads past column WB-1 are zero.  Returns the buffer holding the result.
// ---------------------------------------------------------------------------------------
template <int LOGR, int WB, int NT>
__device__ __forceinline__ float* fht_stages_smem(float* cur, float* nxt)
{
    constexpr int R = 1 << LOGR;
#pragma unroll 1
    for (int s = 1; s <= LOGR; ++s) {
        const int h = 1 << (s - 1);
        for (int idx = threadIdx.x; idx < (R / 2) * WB; idx += NT) {
            const int pr = idx / WB;
            const int x = idx - pr * WB;
            const int lo = pr & (h - 1);
            const int r = ((pr >> (s - 1)) << s) | lo;
            const int t = rev_bits(lo, s - 1);
            const float a = cur[r * WB + x];
            const int xb = x + t;
            const float b0 = (xb < WB) ? cur[(r + h) * WB + xb] : 0.0f;
            const float b1 = (xb + 1 < WB) ? cur[(r + h) * WB + xb + 1] : 0.0f;
            nxt[r * WB + x] = a + b0;
            nxt[(r + h) * WB + x] = a + b1;
        }
        __syncthreads();
        float* tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    return cur;
}

struct Pass1Args {
    const float* src;       // filtered sinogram [count][K][M] or linogram [count][4][N][2N]
    float* g;               // [count][4][N][2N]
    const RowGeom* geom;
    int N, K, M;
    int n1;
};

// Pass 1: CTA = (column tile, quarter * blocks + block, slice).  Loads (or resamples) the
// block's 2^LOGR linogram rows over the tile plus halo, runs LOGR stages, writes G.
template <int LOGR, bool FROM_LIN>
__global__ void __launch_bounds__(kP1Threads)
pass1_kernel(Pass1Args a)
{
    constexpr int R = 1 << LOGR;
    constexpr int T = kP1Tile;
    constexpr int WB = T + R;
    extern __shared__ float smem[];
    float* buf0 = smem;
    float* buf1 = smem + R * WB;

    const int N = a.N, W = 2 * N;
    const int nblocks = N >> LOGR;
    const int q = blockIdx.y / nblocks;
    const int bi = blockIdx.y - q * nblocks;
    const int s = blockIdx.z;
    const int c0 = blockIdx.x * T;
    if (c0 >= N + R * bi) return;                      // nothing needed in this tile

    const size_t lin_q = ((size_t)s * 4 + q) * N;      // row index base of this quarter
    for (int idx = threadIdx.x; idx < R * WB; idx += kP1Threads) {
        const int j = idx / WB;
        const int x = idx - j * WB;
        const int i = bi * R + j;
        const int c = c0 + x;
        float v = 0.0f;
        if (c <= N - 1 + i && c < W) {
            if (FROM_LIN) {
                v = a.src[(lin_q + i) * W + c];
            } else {
                const RowGeom gm = a.geom[q * N + i];
                v = linogram_sample(gm, a.src + (size_t)s * a.K * a.M, a.K, a.M, c);
            }
        }
        buf0[idx] = v;
    }
    __syncthreads();
    const float* res = fht_stages_smem<LOGR, WB, kP1Threads>(buf0, buf1);

    for (int idx = threadIdx.x; idx < R * T; idx += kP1Threads) {
        const int j = idx / T;
        const int x = idx - j * T;
        const int tau = rev_bits(j, LOGR);
        const int c = c0 + x;
        if (c < N + (tau + 1) * bi)
            a.g[(lin_q + (size_t)bi * R + tau) * W + c] = res[j * WB + x];
    }
}

struct Pass2Args {
    const float* g;         // [count][4][N][2N]
    float* img;             // [count][N][N]
    int N, n1;
};

// Pass 2 + quarter sum: CTA = (image tile x, image tile y, slice).  For each quarter and
// each slope group tau_hi covering the tile, loads the sheared G rows, runs LOGR2 stages
// and scatters the quarter image into the tile: v quarters as [y][x], h quarters
// transposed, '+' quarters mirrored.  f = (F_v- + F_v+) + (F_h- + F_h+).
template <int LOGR2>
__global__ void __launch_bounds__(kP2Threads)
pass2_kernel(Pass2Args a)
{
    constexpr int R2 = 1 << LOGR2;
    constexpr int TL = kP2Tile;
    constexpr int WB = TL + R2;
    constexpr int TP = TL + 1;               // padded tile row
    extern __shared__ float smem[];
    float* buf0 = smem;
    float* buf1 = buf0 + R2 * WB;
    float* sv = buf1 + R2 * WB;              // [TL][TP]  F_v- + F_v+
    float* sh = sv + TL * TP;                // [TL][TP]  F_h- + F_h+

    const int N = a.N, W = 2 * N;
    const int R1 = 1 << a.n1;
    const int x0 = blockIdx.x * TL;
    const int y0 = blockIdx.y * TL;
    const int s = blockIdx.z;

    for (int q = 0; q < 4; ++q) {
        const float* gq = a.g + ((size_t)s * 4 + q) * N * W;
        const int tau_base = (q < 2) ? y0 : x0;
        int uo;
        if (q == 0) uo = x0;
        else if (q == 1) uo = N - x0 - TL;
        else if (q == 2) uo = y0;
        else uo = N - y0 - TL;
        for (int grp = 0; grp < TL / R2; ++grp) {
            const int tau_hi = tau_base / R2 + grp;
            for (int idx = threadIdx.x; idx < R2 * WB; idx += kP2Threads) {
                const int ih = idx / WB;
                const int x = idx - ih * WB;
                const int col = uo + tau_hi * ih + x;
                float v = 0.0f;
                if (col < N + (tau_hi + 1) * ih)
                    v = gq[((size_t)ih * R1 + tau_hi) * W + col];
                buf0[idx] = v;
            }
            __syncthreads();
            const float* res = fht_stages_smem<LOGR2, WB, kP2Threads>(buf0, buf1);
            for (int idx = threadIdx.x; idx < R2 * TL; idx += kP2Threads) {
                const int j = idx / TL;
                const int xx = idx - j * TL;
                const int t = grp * R2 + rev_bits(j, LOGR2);   // tau - tau_base
                const float v = res[j * WB + xx];
                if (q == 0) sv[t * TP + xx] = v;
                else if (q == 1) sv[t * TP + (TL - 1 - xx)] += v;
                else if (q == 2) sh[xx * TP + t] = v;
                else sh[(TL - 1 - xx) * TP + t] += v;
            }
            __syncthreads();
        }
    }
    float* out = a.img + (size_t)s * N * N;
    for (int idx = threadIdx.x; idx < TL * TL; idx += kP2Threads) {
        const int yy = idx / TL;
        const int xx = idx - yy * TL;
        out[(size_t)(y0 + yy) * N + x0 + xx] = sv[yy * TP + xx] + sh[yy * TP + xx];
    }
}

// Single-pass sizes (n <= 6): G already holds the quarter images H_q[tau][u]; sum them.
__global__ void __launch_bounds__(256)
combine_kernel(const float* __restrict__ g, float* __restrict__ img, int N)
{
    const int W = 2 * N;
    const int s = blockIdx.y;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N * N) return;
    const int y = p / N;
    const int x = p - y * N;
    const float* h = g + (size_t)s * 4 * N * W;
    const size_t qs = (size_t)N * W;
    const float v = h[(size_t)y * W + x] + h[qs + (size_t)y * W + (N - 1 - x)];
    const float hh = h[2 * qs + (size_t)x * W + y] + h[3 * qs + (size_t)x * W + (N - 1 - y)];
    img[(size_t)s * N * N + p] = v + hh;
}

template <int LOGR, bool FROM_LIN>
size_t pass1_smem() { return (size_t)2 * (1 << LOGR) * (kP1Tile + (1 << LOGR)) * sizeof(float); }

template <int LOGR2>
size_t pass2_smem()
{
    return ((size_t)2 * (1 << LOGR2) * (kP2Tile + (1 << LOGR2)) + 2 * kP2Tile * (kP2Tile + 1)) *
           sizeof(float);
}

template <int LOGR, bool FROM_LIN>
cudaError_t launch_pass1_t(const fbp_plan_s* p, const float* src, float* g, int count,
                           cudaStream_t st)
{
    const int R = 1 << LOGR;
    const int nblocks = p->N >> LOGR;
    const int max_cols = p->N + R * (nblocks - 1);
    dim3 grid((max_cols + kP1Tile - 1) / kP1Tile, 4 * nblocks, count);
    Pass1Args a{src, g, p->d_geom, p->N, p->K, p->M, p->n1};
    pass1_kernel<LOGR, FROM_LIN><<<grid, kP1Threads, pass1_smem<LOGR, FROM_LIN>(), st>>>(a);
    return cudaGetLastError();
}

template <int LOGR2>
cudaError_t launch_pass2_t(const fbp_plan_s* p, const float* g, float* img, int count,
                           cudaStream_t st)
{
    dim3 grid(p->N / kP2Tile, p->N / kP2Tile, count);
    Pass2Args a{g, img, p->N, p->n1};
    pass2_kernel<LOGR2><<<grid, kP2Threads, pass2_smem<LOGR2>(), st>>>(a);
    return cudaGetLastError();
}

template <int LOGR, bool FROM_LIN>
cudaError_t set_p1_attr()
{
    return cudaFuncSetAttribute(pass1_kernel<LOGR, FROM_LIN>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)pass1_smem<LOGR, FROM_LIN>());
}

template <int LOGR2>
cudaError_t set_p2_attr()
{
    return cudaFuncSetAttribute(pass2_kernel<LOGR2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)pass2_smem<LOGR2>());
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
#define FBP_P2(L) \
    if (e == cudaSuccess) e = set_p2_attr<L>();
    FBP_P2(1) FBP_P2(2) FBP_P2(3) FBP_P2(4) FBP_P2(5) FBP_P2(6)
#undef FBP_P2
    return e;
}

cudaError_t launch_resample(const fbp_plan_s* p, const float* filt, float* lin, int count,
                            cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    dim3 grid((2 * p->N + 255) / 256, 4 * p->N, count);
    resample_kernel<<<grid, 256, 0, st>>>(filt, lin, p->d_geom, p->N, p->K, p->M);
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
                         cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    if (p->n2 == 0) {
        dim3 grid((p->N * p->N + 255) / 256, count);
        combine_kernel<<<grid, 256, 0, st>>>(g, img, p->N);
        return cudaGetLastError();
    }
    switch (p->n2) {
        case 1: return launch_pass2_t<1>(p, g, img, count, st);
        case 2: return launch_pass2_t<2>(p, g, img, count, st);
        case 3: return launch_pass2_t<3>(p, g, img, count, st);
        case 4: return launch_pass2_t<4>(p, g, img, count, st);
        case 5: return launch_pass2_t<5>(p, g, img, count, st);
        case 6: return launch_pass2_t<6>(p, g, img, count, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fbp
