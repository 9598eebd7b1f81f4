// Recursive ramp filtering of every projection row (paper Sec. 3, Eq. 9, 12, 13).
//
//   y(n) = sum_{k<mb} b_k p(n-k) - sum_{k=1..q} a_k y(n-k)      causal, n = 0..M-1
//   z(n) = sum_{k<mb} b_k p(n+k) - sum_{k=1..q} a_k z(n+k)      anticausal, n = M-1..0
//   out(n) = y(n) + z(n)                                         zero state outside [0, M)
//
// The plan hands the kernel the same transfer function in parallel form,
//   y(n) = sum_j Re(r_j s_j(n)) + sum_k d_k p(n-k),   s_j(n) = p_j s_j(n-1) + p(n),
// which stays accurate in float32 where the direct form does not (its poles crowd z = 1).
//
// One warp filters one row.  The row is staged in shared memory with coalesced loads;
// lane j owns the contiguous chunk [jL, jL+L) (L odd, so the lanes' strided shared-memory
// accesses fall in 32 distinct banks).  Each mode is a first-order linear recurrence, so
// each direction runs as a blocked scan:
//   1. every lane runs its chunk from zero state and keeps the end state e_j;
//   2. a Kogge-Stone scan over the 32 lanes composes S_{j+1} = p^L S_j + e_j with the
//      host-precomputed powers p^(L 2^d);
//   3. every lane reruns its chunk from its true incoming state and emits the output.
// The causal result is parked in a second shared buffer, the anticausal result is added
// to it, and the row is written back with coalesced stores: one HBM read and one HBM
// write per sample for both directions.
#include "fbp_internal.h"

namespace fbp {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxSmem = 227 * 1024;     // shared memory per CTA on sm_103a

template <int JR, int JC>
struct ModeState {
    float r[JR > 0 ? JR : 1];
    float cr[JC > 0 ? JC : 1];
    float ci[JC > 0 ? JC : 1];
};

template <int JR, int JC>
__device__ __forceinline__ void zero_state(ModeState<JR, JC>& s)
{
#pragma unroll
    for (int j = 0; j < JR; ++j) s.r[j] = 0.0f;
#pragma unroll
    for (int j = 0; j < JC; ++j) { s.cr[j] = 0.0f; s.ci[j] = 0.0f; }
}

// s <- p s + x for every mode
template <int JR, int JC>
__device__ __forceinline__ void step(ModeState<JR, JC>& s, const IirParams& prm, float x)
{
#pragma unroll
    for (int j = 0; j < JR; ++j) s.r[j] = fmaf(prm.rp[j], s.r[j], x);
#pragma unroll
    for (int j = 0; j < JC; ++j) {
        const float nr = fmaf(prm.cpr[j], s.cr[j], fmaf(-prm.cpi[j], s.ci[j], x));
        const float ni = fmaf(prm.cpi[j], s.cr[j], prm.cpr[j] * s.ci[j]);
        s.cr[j] = nr;
        s.ci[j] = ni;
    }
}

// sum_j Re(r_j s_j)
template <int JR, int JC>
__device__ __forceinline__ float output(const ModeState<JR, JC>& s, const IirParams& prm)
{
    float y = 0.0f;
#pragma unroll
    for (int j = 0; j < JR; ++j) y = fmaf(prm.rr[j], s.r[j], y);
#pragma unroll
    for (int j = 0; j < JC; ++j) y = fmaf(prm.crr[j], s.cr[j], fmaf(-prm.cri[j], s.ci[j], y));
    return y;
}

template <bool FORWARD>
__device__ __forceinline__ float shfl(float v, int off)
{
    return FORWARD ? __shfl_up_sync(kFull, v, off) : __shfl_down_sync(kFull, v, off);
}

// Exclusive scan of the lanes' end states: on return s holds the state entering this
// lane's chunk (from lower lanes if FORWARD, from higher lanes otherwise).
template <int JR, int JC, bool FORWARD>
__device__ __forceinline__ void carry_scan(ModeState<JR, JC>& s, const IirParams& prm, int lane)
{
#pragma unroll
    for (int d = 0; d < kScanSteps; ++d) {
        const int off = 1 << d;
        const bool take = FORWARD ? (lane >= off) : (lane + off < 32);
#pragma unroll
        for (int j = 0; j < JR; ++j) {
            const float u = shfl<FORWARD>(s.r[j], off);
            if (take) s.r[j] = fmaf(prm.rpow[d][j], u, s.r[j]);
        }
#pragma unroll
        for (int j = 0; j < JC; ++j) {
            const float ur = shfl<FORWARD>(s.cr[j], off);
            const float ui = shfl<FORWARD>(s.ci[j], off);
            if (take) {
                const float pr = prm.cpowr[d][j], pi = prm.cpowi[d][j];
                s.cr[j] = fmaf(pr, ur, fmaf(-pi, ui, s.cr[j]));
                s.ci[j] = fmaf(pi, ur, fmaf(pr, ui, s.ci[j]));
            }
        }
    }
    const bool edge = FORWARD ? (lane == 0) : (lane == 31);
#pragma unroll
    for (int j = 0; j < JR; ++j) {
        const float u = shfl<FORWARD>(s.r[j], 1);
        s.r[j] = edge ? 0.0f : u;
    }
#pragma unroll
    for (int j = 0; j < JC; ++j) {
        const float ur = shfl<FORWARD>(s.cr[j], 1);
        const float ui = shfl<FORWARD>(s.ci[j], 1);
        s.cr[j] = edge ? 0.0f : ur;
        s.ci[j] = edge ? 0.0f : ui;
    }
}

template <int JR, int JC>
__global__ void __launch_bounds__(128)
iir_ramp_kernel(const float* in, float* out, int rows, int M, int warps_per_cta, IirParams prm)
{
    extern __shared__ float smem[];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const long long row = (long long)blockIdx.x * warps_per_cta + warp;
    if (warp >= warps_per_cta || row >= rows) return;     // whole warps leave together

    float* sp = smem + (size_t)warp * 2 * M;              // input row
    float* sy = sp + M;                                    // result row
    const float* src = in + row * (long long)M;
    // every element of the row in flight at once: asynchronous 4-byte copies into shared
    for (int n = lane; n < M; n += 32) {
        const unsigned d = (unsigned)__cvta_generic_to_shared(sp + n);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src + n) : "memory");
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncwarp();

    const int L = prm.L;
    const int n0 = min(lane * L, M);
    const int n1 = min(n0 + L, M);
    const int nd = prm.nd;
    ModeState<JR, JC> s;
    // The recurrences read the chunk in blocks of kB samples fetched ahead into registers,
    // so shared-memory latency stays off the dependency chain.
    constexpr int kB = 8;
    auto causal_out = [&](int n) {
        float y = output(s, prm);
        for (int k = 0; k < nd; ++k)
            if (n - k >= 0) y = fmaf(prm.d[k], sp[n - k], y);
        sy[n] = y;
    };
    auto anticausal_out = [&](int n) {
        float z = output(s, prm);
        for (int k = 0; k < nd; ++k)
            if (n + k < M) z = fmaf(prm.d[k], sp[n + k], z);
        sy[n] += z;
    };

    // causal: local pass from zero state, carry scan, final pass
    zero_state(s);
    int n = n0;
    for (; n + kB <= n1; n += kB) {
        float x[kB];
#pragma unroll
        for (int k = 0; k < kB; ++k) x[k] = sp[n + k];
#pragma unroll
        for (int k = 0; k < kB; ++k) step(s, prm, x[k]);
    }
    for (; n < n1; ++n) step(s, prm, sp[n]);
    carry_scan<JR, JC, true>(s, prm, lane);
    n = n0;
    for (; n + kB <= n1; n += kB) {
        float x[kB];
#pragma unroll
        for (int k = 0; k < kB; ++k) x[k] = sp[n + k];
#pragma unroll
        for (int k = 0; k < kB; ++k) {
            step(s, prm, x[k]);
            causal_out(n + k);
        }
    }
    for (; n < n1; ++n) {
        step(s, prm, sp[n]);
        causal_out(n);
    }

    // anticausal: the same, walking the chunk backwards
    zero_state(s);
    n = n1 - 1;
    for (; n - kB + 1 >= n0; n -= kB) {
        float x[kB];
#pragma unroll
        for (int k = 0; k < kB; ++k) x[k] = sp[n - k];
#pragma unroll
        for (int k = 0; k < kB; ++k) step(s, prm, x[k]);
    }
    for (; n >= n0; --n) step(s, prm, sp[n]);
    carry_scan<JR, JC, false>(s, prm, lane);
    n = n1 - 1;
    for (; n - kB + 1 >= n0; n -= kB) {
        float x[kB];
#pragma unroll
        for (int k = 0; k < kB; ++k) x[k] = sp[n - k];
#pragma unroll
        for (int k = 0; k < kB; ++k) {
            step(s, prm, x[k]);
            anticausal_out(n - k);
        }
    }
    for (; n >= n0; --n) {
        step(s, prm, sp[n]);
        anticausal_out(n);
    }
    __syncwarp();

    float* dst = out + row * (long long)M;
    for (int n = lane; n < M; n += 32) dst[n] = sy[n];
}

template <int JR, int JC>
cudaError_t launch_iir_t(const fbp_plan_s* p, const float* in, float* out, int rows,
                         cudaStream_t st)
{
    const size_t per_warp = (size_t)2 * p->M * sizeof(float);
    int warps = (int)(kMaxSmem / per_warp);
    warps = warps > 4 ? 4 : warps;
    if (warps < 1) return cudaErrorInvalidValue;
    const size_t smem = per_warp * warps;
    const int grid = (rows + warps - 1) / warps;
    iir_ramp_kernel<JR, JC><<<grid, 128, smem, st>>>(in, out, rows, p->M, warps, p->iir);
    return cudaGetLastError();
}

template <int JR, int JC>
cudaError_t set_attr()
{
    return cudaFuncSetAttribute(iir_ramp_kernel<JR, JC>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
}

// Every (real modes, complex modes) split with jr + 2 jc <= 8.
#define FBP_IIR_MODES(X)                                                              \
    X(0, 0) X(1, 0) X(2, 0) X(3, 0) X(4, 0) X(5, 0) X(6, 0) X(7, 0) X(8, 0)          \
    X(0, 1) X(1, 1) X(2, 1) X(3, 1) X(4, 1) X(5, 1) X(6, 1)                          \
    X(0, 2) X(1, 2) X(2, 2) X(3, 2) X(4, 2)                                          \
    X(0, 3) X(1, 3) X(2, 3) X(0, 4)

}  // namespace

cudaError_t prepare_iir_kernels()
{
    cudaError_t e = cudaSuccess;
#define FBP_X(R, C) \
    if (e == cudaSuccess) e = set_attr<R, C>();
    FBP_IIR_MODES(FBP_X)
#undef FBP_X
    return e;
}

cudaError_t launch_iir(const fbp_plan_s* p, const float* in, float* out, int rows,
                       cudaStream_t st)
{
    if (rows <= 0) return cudaSuccess;
    const int jr = p->iir.jr, jc = p->iir.jc;
#define FBP_X(R, C) \
    if (jr == R && jc == C) return launch_iir_t<R, C>(p, in, out, rows, st);
    FBP_IIR_MODES(FBP_X)
#undef FBP_X
    return cudaErrorInvalidValue;
}

}  // namespace fbp
