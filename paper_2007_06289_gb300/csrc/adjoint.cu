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
// and ending with L-bar[i][c] = A_0[i][0][c].  Up to five stages run per launch in shared
// memory (below), over all slices and quarters, ping-ponging between two [count][4][N][2N]
// buffers; every output element is one fixed float32 sum, so the result is reproducible bit
// for bit.
//
// Resampling, transposed.  Each linogram sample is w0 * lerp(row k0) + w1 * lerp(row k1)
// (Eq. 14-15 with the float32 weights the forward kernels use); its transpose adds the
// sample's gradient times the four bilinear weights into the sinogram gradient, gathered
// per detector bin in a fixed order (reproducible bit for bit).
#include "fbp_internal.h"

namespace fbp {
namespace {

constexpr int kAdjThreads = 256;
constexpr int kAfMaxStages = 5;

// ---------------------------------------------------------------- fused transposed stages
// One launch runs S consecutive transposed stages, level k -> level k - S, in shared memory.
//
// Groups.  Output strip b 2^S + C (C in [0, 2^S)), slope t at level k - S depends only on the
// 2^S consecutive level-k rows b 2^k + 2^S t + j of strip b: unrolling the stage formula S
// times,
//     A_{k-S}[b 2^S + C][t][v] = sum_j A_k[b][2^S t + j][v - C t - s(C, j)],
// the shift splitting into C t (C read with its first stage's bit highest) and a small part
// s(C, j) in [0, 2^S - 1] that is exactly the shift of the same S stages run on the 2^S rows
// alone (slope t = 0).  A CTA therefore loads its group's 2^S rows over a tile of columns
// x plus a halo of 2^S - 1, runs the S stages on them in shared memory with the small
// slopes, and writes output row C at column x + C t (a skewed tile).  Each output is the same
// float32 sum in the same order as one launch per stage: the result is reproducible bit for
// bit, and equal to the stage-by-stage recursion.
//
// Written ranges.  Level-k row (b, tau) can be non-zero only on columns
// [b tau, b tau + N + 2^(n-k) - 1) (its inputs are image columns [0, N) moved right by
// b tau plus at most 2^(n-k) - 1).  Each launch computes and writes exactly that range of
// its output rows (clipped to the row width W = 2N), and reads its input rows as zero outside
// theirs, so the level arrays between launches are never cleared; the last launch (level 0,
// the linogram gradient) writes every column.
template <int S> constexpr int af_halo() { return ((1 << S) - 1 + 3) & ~3; }
constexpr int kAfCols = kAdjThreads;            // shared-memory columns: one per thread
template <int S> constexpr int af_tile() { return kAfCols - af_halo<S>(); }
constexpr int kAfPitch = kAfCols + 1;           // odd: conflict-free column-wise writes
template <int S> constexpr size_t af_smem() { return 2 * (size_t)(1 << S) * kAfPitch * sizeof(float); }

// RESID (last launch only): the output is turned into the SIRT residual on the way out,
// (b - out) * rinv, b [count][4][N][2N] and rinv one slice's [4][N][2N].  `in` holds in_n
// floats and `out` out_n (b: out_n, rinv: out_n / count); in the bounds-checked build every
// global index is tested against them.
template <int S, bool FROM_IMAGE, bool RESID>
__global__ void __launch_bounds__(kAdjThreads)
adj_fused_kernel(const float* __restrict__ in, float* __restrict__ out, int N, int n, int k,
                 int wc, const float* __restrict__ rb, const float* __restrict__ rw,
                 long long in_n, long long out_n, long long rw_n, int* status)
{
    constexpr int R = 1 << S;
    constexpr int H = af_halo<S>();
    constexpr int T = af_tile<S>();
    extern __shared__ float sm[];
    const int W = 2 * N;
    const int tid = threadIdx.x;
    const int sq = blockIdx.z;                  // slice * 4 + quarter
    const int ko = k - S;                       // output level
    const int g = blockIdx.y;                   // group: input rows g 2^S + j of level k
    const int b = g >> ko, t = g & ((1 << ko) - 1);
    const int xa = (b * t) << S;                // first column of every output row's range
    const int x0 = xa + blockIdx.x * T;         // first output column (before the C t skew)
    if (x0 >= W) return;                        // every output column x + C t >= W
    const int xs = x0 - H;                      // column of shared column 0
    const Span si{in, in_n, status};

    // load the group's rows: shared row j, column p <-> input column xs + p
    float* X = sm;
    if constexpr (FROM_IMAGE) {
        // level n = the quarter gradients of Eq. 22's index maps (g = t here, b = 0):
        // v-: G[tau][u]  v+: G[tau][N-1-u]  h-: G[u][tau]  h+: G[N-1-u][tau], zero for u >= N
        const float* gi = in + (size_t)(sq >> 2) * N * N;
        const int q = sq & 3;
        const int tau0 = g << S;
        if (q < 2) {
            const int x = xs + tid;
            const bool ok = x >= 0 && x < N;
            const int u = q == 0 ? x : N - 1 - x;
            float v[R];                         // all of the rows' loads in flight at once
#pragma unroll
            for (int j = 0; j < R; ++j) v[j] = ok ? ld_in(si, gi + (size_t)(tau0 + j) * N + u) : 0.0f;
#pragma unroll
            for (int j = 0; j < R; ++j) X[j * kAfPitch + tid] = v[j];
        } else {
            // columns of G: j fastest so that the 2^S rows' values of one u are adjacent
            float v[R];
#pragma unroll
            for (int it = 0; it < R; ++it) {
                const int idx = tid + it * kAdjThreads;
                const int j = idx & (R - 1);
                const int x = xs + (idx >> S);
                const bool ok = x >= 0 && x < N;
                const int u = q == 2 ? x : N - 1 - x;
                v[it] = ok ? ld_in(si, gi + (size_t)u * N + tau0 + j) : 0.0f;
            }
#pragma unroll
            for (int it = 0; it < R; ++it) {
                const int idx = tid + it * kAdjThreads;
                X[(idx & (R - 1)) * kAfPitch + (idx >> S)] = v[it];
            }
        }
    } else {
        const float* rows = in + ((size_t)sq * N + ((size_t)g << S)) * W;
        const int span = N + (1 << (n - k)) - 1;   // written length of every level-k row
        const int x = xs + tid;
        float v[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int lo = xa + b * j;          // b (2^S t + j)
            const int hi = min(W, lo + span);
            v[j] = (x >= lo && x < hi) ? ld_in(si, rows + (size_t)j * W + x) : 0.0f;
        }
#pragma unroll
        for (int j = 0; j < R; ++j) X[j * kAfPitch + tid] = v[j];
    }
    // RESID: the last launch (t = 0, so output row C lands at column x itself); start this
    // thread's data and weight loads now so that they arrive during the stage sweeps
    float rbv[RESID ? R : 1], rwv[RESID ? R : 1];
    if constexpr (RESID) {
        const int x = xs + tid;
        const bool ok = tid >= H && x < xa + wc && x < W;
        const size_t o = ((size_t)sq * N + ((size_t)b << S)) * W + x;
        const size_t ow = o - (size_t)(sq >> 2) * 4 * N * W;
        const Span sb{rb, out_n, status}, sw{rw, rw_n, status};
#pragma unroll
        for (int C = 0; C < R; ++C) {
            rbv[C] = ok ? ld_in(sb, rb + o + (size_t)C * W) : 0.0f;
            rwv[C] = ok ? ld_in(sw, rw + ow + (size_t)C * W) : 0.0f;
        }
    }
    __syncthreads();

    // S transposed stages on the 2^S rows (slopes of the group alone), ping-ponging between
    // the two shared buffers; row bc 2^(m-1) + tl of level m-1 from rows bl 2^m + 2tl and
    // bl 2^m + 2tl + 1 of level m, bl = bc / 2.  Columns below 0 read as zero (they only
    // feed halo columns).
    float* cur = X;
    float* nxt = X + R * kAfPitch;
    const int p = tid;
#pragma unroll
    for (int m = S; m >= 1; --m) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int bc = r >> (m - 1), tl = r & ((1 << (m - 1)) - 1);
            const float* a0 = cur + (((bc >> 1) << m) + 2 * tl) * kAfPitch;
            const float* a1 = a0 + kAfPitch;
            float o;
            if ((bc & 1) == 0) {
                o = a0[p] + a1[p];
            } else {
                const float y0 = p >= tl ? a0[p - tl] : 0.0f;
                const float y1 = p >= tl + 1 ? a1[p - tl - 1] : 0.0f;
                o = y0 + y1;
            }
            nxt[r * kAfPitch + p] = o;
        }
        __syncthreads();
        float* sw = cur;
        cur = nxt;
        nxt = sw;
    }

    // shared row C = output strip b 2^S + C, slope t: column x = xs + p goes to x + C t,
    // for x below the end of the written range xa + wc
    if (p >= H) {
        const int x = xs + p;
        const Span so{out, out_n, status};
        if (x < xa + wc) {
            const size_t o = ((size_t)sq * N + ((size_t)b << (S + ko)) + t) * W + x;
#pragma unroll
            for (int C = 0; C < R; ++C) {
                const int v = x + C * t;
                if (v < W) {
                    const size_t oc = o + ((size_t)C << ko) * W + (size_t)C * t;
                    float val = cur[C * kAfPitch + p];
                    if constexpr (RESID) val = (rbv[C] - val) * rwv[C];
                    if (so.ok(out + oc)) out[oc] = val;
                }
            }
        }
    }
}

template <int S>
cudaError_t set_af_attr()
{
    const int bytes = (int)af_smem<S>();
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(adj_fused_kernel<S, true, false>, a, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(adj_fused_kernel<S, false, false>, a, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(adj_fused_kernel<S, true, true>, a, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(adj_fused_kernel<S, false, true>, a, bytes);
    return e;
}

template <int S>
cudaError_t launch_af(const float* in, float* out, int N, int n, int k, int count, bool from_image,
                      const float* rb, const float* rw, int* status, cudaStream_t st)
{
    const int W = 2 * N;
    const long long lin_n = (long long)count * 4 * N * W;
    const long long in_n = from_image ? (long long)count * N * N : lin_n;
    const long long rw_n = (long long)4 * N * W;
    // written length of every output row: the last launch (level 0) writes all W columns
    const int wc = k == S ? W : N + (1 << (n - k + S)) - 1;
    const dim3 grid((wc + af_tile<S>() - 1) / af_tile<S>(), N >> S, 4 * count);
    const size_t sm = af_smem<S>();
    const bool resid = rb != nullptr && k == S;
    if (from_image && resid)
        adj_fused_kernel<S, true, true><<<grid, kAdjThreads, sm, st>>>(in, out, N, n, k, wc, rb, rw,
                                                                          in_n, lin_n, rw_n, status);
    else if (from_image)
        adj_fused_kernel<S, true, false><<<grid, kAdjThreads, sm, st>>>(in, out, N, n, k, wc, rb, rw,
                                                                          in_n, lin_n, rw_n, status);
    else if (resid)
        adj_fused_kernel<S, false, true><<<grid, kAdjThreads, sm, st>>>(in, out, N, n, k, wc, rb, rw,
                                                                          in_n, lin_n, rw_n, status);
    else
        adj_fused_kernel<S, false, false><<<grid, kAdjThreads, sm, st>>>(in, out, N, n, k, wc, rb, rw,
                                                                          in_n, lin_n, rw_n, status);
    return cudaGetLastError();
}

// Transposed resampling as a gather: a CTA owns kRsRows consecutive sinogram rows of one
// slice, a thread 4 consecutive bins j0..j0+3 of each.  The plan lists the linogram rows
// whose resampling reads the group's rows (each with its weight into every row of the
// group: w0 into its angle row k0, w1 into k0 + 1, or into row 0 with the detector
// mirrored, m' = M - 1 - m, past the last angle).  For each listed row the thread walks the
// columns c whose detector position m(c) = a c + b (32.32 fixed point, monotone in c,
// |a| <= 1) falls in [j0 - 1, j0 + 4), tests each exactly, and sums L-bar[c] (1 - f) into
// bin floor(m) and L-bar[c] f into bin floor(m) + 1 where those are its own (the forward
// resampling's positions and float32 fractions); the row's sums then go to every group row
// it reads, times that row's weight.  Computing each linogram row's sums once for both of
// its angle rows is what grouping the rows saves.  No atomics: the order of the additions
// is fixed (table order, c ascending), so the result is reproducible bit for bit.
constexpr int kRsEnt = 32;                      // reader rows staged per round
constexpr int kRsBins = 4;                      // bins per thread (s0 .. s3)
constexpr int kRsWin = 10;                      // columns a thread reads per reader row

// count slices; in the bounds-checked build every global index (the tables' included) is
// tested against its buffer.
__global__ void __launch_bounds__(kAdjThreads, 1)
adj_resample_kernel(const float* __restrict__ lbar, float* __restrict__ pbar,
                    const RowGeom* __restrict__ geom, const int* __restrict__ rptr,
                    const ReaderEntry* __restrict__ rent, int N, int K, int M, int count,
                    int n_ent, int* status)
{
    __shared__ long long ea[kRsEnt], eb[kRsEnt];    // m(c) = ea c + eb (mirror folded in)
    __shared__ float efi[kRsEnt], efb[kRsEnt];      // 1 / a and b in float, for the estimate
    __shared__ float4 ew[kRsEnt];                   // weights into the group's rows
    __shared__ int eq[kRsEnt];
    static_assert(kRsRows == 4, "weights staged as float4");
    const int grp = blockIdx.y;
    const int s = blockIdx.z;
    const int W = 2 * N;
    const int j0 = (blockIdx.x * kAdjThreads + threadIdx.x) * kRsBins;
    const float* ls = lbar + (size_t)s * 4 * N * W;
    const Span sl{lbar, (long long)count * 4 * N * W, status};
    const Span sp{pbar, (long long)count * K * M, status};
    float acc[kRsRows][kRsBins];
#pragma unroll
    for (int r = 0; r < kRsRows; ++r)
#pragma unroll
        for (int b = 0; b < kRsBins; ++b) acc[r][b] = 0.0f;
    const int ngrp = (K + kRsRows - 1) / kRsRows;
    const int r0 = in_bounds(status, grp, ngrp) ? rptr[grp] : 0;
    const int r1 = in_bounds(status, grp, ngrp) ? rptr[grp + 1] : 0;
    for (int rb = r0; rb < r1; rb += kRsEnt) {
        const int ne = min(kRsEnt, r1 - rb);
        __syncthreads();                        // previous round's tables are read
        if (threadIdx.x < ne) {
            ReaderEntry en = {0, {0.0f, 0.0f, 0.0f, 0.0f}};
            if (in_bounds(status, rb + threadIdx.x, n_ent)) en = rent[rb + threadIdx.x];
            const int qi = in_bounds(status, en.code >> 1, 4LL * N) ? en.code >> 1 : 0;
            const RowGeom gm = geom[qi];
            long long a = gm.a_fx, b = gm.b_fx;
            if (en.code & 1) {                  // m' = (M - 1) - m = -a c + ((M - 1) - b)
                b = ((long long)(M - 1) << kFixBits) - b;
                a = -a;
            }
            ea[threadIdx.x] = a;
            eb[threadIdx.x] = b;
            efi[threadIdx.x] = __fdividef(1.0f, (float)a * 0x1p-32f);   // estimate only
            efb[threadIdx.x] = (float)b * 0x1p-32f;
            ew[threadIdx.x] = make_float4(en.w[0], en.w[1], en.w[2], en.w[3]);
            eq[threadIdx.x] = qi;
        }
        __syncthreads();
        if (j0 >= M) continue;
        for (int e = 0; e < ne; ++e) {
            const float fi = efi[e], fb = efb[e];
            // columns with m(c) in [j0 - 1, j0 + 4): an interval of 5 / |a| <= 5 sqrt 2
            // columns (|a| >= 1 / sqrt 2), so at most 8 of them; the float estimate of the
            // first may land one below it: a window of kRsWin = 10 from floor(estimate),
            // loaded all at once (checked over every row and bin group for N = 256 .. 4096)
            const float c1 = ((float)(j0 - 1) - fb) * fi;
            const float c2 = ((float)(j0 + kRsBins) - fb) * fi;
            const float clo = fmaxf(fminf(c1, c2), 0.0f);
            const float chi = fminf(fmaxf(c1, c2) + 1.0f, (float)(W - 1));
            if (clo > chi) continue;
            const int cs = (int)clo, ce = (int)chi;
            const long long a = ea[e];
            const float* lr = ls + (size_t)eq[e] * W + cs;
            float lv[kRsWin];
#pragma unroll
            for (int u = 0; u < kRsWin; ++u) lv[u] = cs + u <= ce ? ld_in(sl, lr + u) : 0.0f;
            const long long mb = eb[e] + a * (long long)cs;
            float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;    // bins j0 .. j0 + 3
#pragma unroll
            for (int u = 0; u < kRsWin; ++u) {
                const long long m = mb + a * u;
                const int d = (int)(m >> kFixBits) - j0;       // bin floor(m) - j0
                if (cs + u > ce || d < -1 || d >= kRsBins) continue;
                const float f = __uint2float_rn((unsigned)m) * 0x1p-32f;
                const float v0 = lv[u] * (1.0f - f), v1 = lv[u] * f;   // to bins d, d + 1
                if (d == -1) s0 += v1;
                else if (d == 0) { s0 += v0; s1 += v1; }
                else if (d == 1) { s1 += v0; s2 += v1; }
                else if (d == 2) { s2 += v0; s3 += v1; }
                else s3 += v0;
            }
            const float4 w = ew[e];
            const float wr[kRsRows] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int r = 0; r < kRsRows; ++r) {
                acc[r][0] = fmaf(wr[r], s0, acc[r][0]);
                acc[r][1] = fmaf(wr[r], s1, acc[r][1]);
                acc[r][2] = fmaf(wr[r], s2, acc[r][2]);
                acc[r][3] = fmaf(wr[r], s3, acc[r][3]);
            }
        }
    }
    if (j0 >= M) return;
#pragma unroll
    for (int r = 0; r < kRsRows; ++r) {
        const int k = grp * kRsRows + r;
        if (k >= K) break;
        float* out = pbar + ((size_t)s * K + k) * M + j0;
#pragma unroll
        for (int b = 0; b < kRsBins; ++b)
            if (j0 + b < M && sp.ok(out + b)) out[b] = acc[r][b];
    }
}

}  // namespace

cudaError_t prepare_adjoint_kernels()
{
    cudaError_t e = set_af_attr<1>();
    if (e == cudaSuccess) e = set_af_attr<2>();
    if (e == cudaSuccess) e = set_af_attr<3>();
    if (e == cudaSuccess) e = set_af_attr<4>();
    if (e == cudaSuccess) e = set_af_attr<5>();
    return e;
}

cudaError_t launch_fht_adjoint(const fbp_plan_s* p, const float* img_grad, float* lin_grad,
                               float* scratch, int count, cudaStream_t st, const float* resid_b,
                               const float* resid_w)
{
    if (count <= 0) return cudaSuccess;
    const int N = p->N, n = p->n;
    // ceil(n / 5) launches of at most five stages each, the larger shares first; start in
    // the buffer that makes the last launch land in lin_grad
    const int launches = (n + kAfMaxStages - 1) / kAfMaxStages;
    float* buf[2] = {lin_grad, scratch};
    int cur = (launches & 1) ? 0 : 1;
    const float* src = img_grad;
    int k = n;
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < launches && e == cudaSuccess; ++l) {
        const int left = launches - l;
        const int S = (k + left - 1) / left;
        switch (S) {
            case 1: e = launch_af<1>(src, buf[cur], N, n, k, count, l == 0, resid_b, resid_w, p->d_status, st); break;
            case 2: e = launch_af<2>(src, buf[cur], N, n, k, count, l == 0, resid_b, resid_w, p->d_status, st); break;
            case 3: e = launch_af<3>(src, buf[cur], N, n, k, count, l == 0, resid_b, resid_w, p->d_status, st); break;
            case 4: e = launch_af<4>(src, buf[cur], N, n, k, count, l == 0, resid_b, resid_w, p->d_status, st); break;
            default: e = launch_af<5>(src, buf[cur], N, n, k, count, l == 0, resid_b, resid_w, p->d_status, st); break;
        }
        src = buf[cur];
        cur ^= 1;
        k -= S;
    }
    return e;
}

cudaError_t launch_resample_adjoint(const fbp_plan_s* p, const float* lin_grad, float* filt_grad,
                                    int count, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    const int per_cta = kAdjThreads * kRsBins;
    const dim3 grid((p->M + per_cta - 1) / per_cta, (p->K + kRsRows - 1) / kRsRows, count);
    adj_resample_kernel<<<grid, kAdjThreads, 0, st>>>(lin_grad, filt_grad, p->d_geom, p->d_readers,
                                                      p->d_reader_ent, p->N, p->K, p->M, count,
                                                      p->n_reader_ent, p->d_status);
    return cudaGetLastError();
}

}  // namespace fbp
