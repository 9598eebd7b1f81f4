// Internal declarations shared by the translation units of libfbp (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "../../include/fbp.h"

namespace fbp {

constexpr int kMaxOrder = FBP_MAX_ORDER;
constexpr int kScanSteps = 5;            // log2(32 lanes)

// Per linogram row (quarter q, slope row i): where the row samples the filtered sinogram.
// Detector index m(c) = A*c + B for stored column c, carried in signed 64-bit fixed point
// with kFixBits = 32 fractional bits: stepping c by one adds a_fx exactly, the bin is the
// high word and the fraction the low word (rounded to float: ~2^-25 absolute accuracy).
// Angle index k0 + ft; the second angle row is k0+1, or row 0 with the detector mirrored
// (m -> M-1-m) when k0+1 == K ("wrap", p(theta+pi, r) = p(theta, -r)).  The row weight w
// (trapezoid in sigma, Jacobian 1/k_t^2) is folded into the angle interpolation weights:
// sample = w1 * p(k0+1, m) + w0 * p(k0, m), w0 = w (1 - ft), w1 = w ft.
constexpr int kFixBits = 32;
struct RowGeom {
    int k0;
    int wrap;
    float w0;
    float w1;
    long long a_fx;
    long long b_fx;
};

// The recursive filter in parallel (modal) form, as the kernel consumes it:
//   g(n) = sum_j Re(r_j p_j^n) + d_n,   i.e.   y(n) = sum_j Re(r_j s_j(n)) + sum_k d_k x(n-k),
//   s_j(n) = p_j s_j(n-1) + x(n).
// jr real modes, jc complex modes (one per conjugate pair, residue doubled), nd direct taps.
// pow*[d] = p^(L 2^d) carries a mode's state across 2^d lanes of L samples each.
// A row is split over wpr warps (32 wpr lanes, L samples per lane): p^(32 L) carries a
// mode's state across one warp.  With diff = 1 the modes are driven by the first
// difference of the input (B(z) = (1 - z^-1) B'(z) when B(1) = 0): DC-free filters then
// need no cancellation between large mode outputs.
struct IirParams {
    int jr, jc, nd, L, wpr, diff;
    float rp[kMaxOrder], rr[kMaxOrder];
    float cpr[kMaxOrder / 2], cpi[kMaxOrder / 2], crr[kMaxOrder / 2], cri[kMaxOrder / 2];
    float rpow[kScanSteps][kMaxOrder];
    float cpowr[kScanSteps][kMaxOrder / 2], cpowi[kScanSteps][kMaxOrder / 2];
    float rwarp[kMaxOrder];
    float cwarpr[kMaxOrder / 2], cwarpi[kMaxOrder / 2];
    float d[kMaxOrder];
};
constexpr int kIirLmax = 23;       // samples per lane (odd: conflict-free strided access)
constexpr int kIirMaxWarps = 32;   // warps per row, so M <= 32 * 32 * 23

}  // namespace fbp

namespace fbp {
// Device status word.  The pipeline's kernels validate the geometry table rows they use
// (always) and, in a build with FBP_BOUNDS_CHECK defined, every global index they form and
// the shared-memory range of every Hough round; a failed check records FBP_ERR_INTERNAL in
// the plan's status word (the first code recorded wins), skips the access (a skipped load
// reads 0, a rejected row is all zeros) and carries on.  fbp_last_device_error reads it.
#ifdef FBP_BOUNDS_CHECK
constexpr bool kBoundsCheck = true;
#else
constexpr bool kBoundsCheck = false;
#endif

__device__ __forceinline__ void flag_status(int* status, int code)
{
    if (status) atomicCAS(status, 0, code);
}

// 0 <= i < n; in the unchecked build always true (and compiled away).
__device__ __forceinline__ bool in_bounds(int* status, long long i, long long n)
{
    if (!kBoundsCheck) return true;
    if (i >= 0 && i < n) return true;
    flag_status(status, (int)FBP_ERR_INTERNAL);
    return false;
}

// A checked region of global memory: loads outside [base, base + n) read 0 and stores there
// are dropped (checked build only; otherwise plain accesses).
struct Span {
    const float* base;
    long long n;
    int* status;
    __device__ __forceinline__ bool ok(const float* p) const { return in_bounds(status, p - base, n); }
};

__device__ __forceinline__ float ldg_in(const Span& s, const float* p)
{
    return s.ok(p) ? __ldg(p) : 0.0f;
}

// The same as a plain load (no read-only cache path): 0 outside the region.
__device__ __forceinline__ float ld_in(const Span& s, const float* p)
{
    return s.ok(p) ? *p : 0.0f;
}

// A geometry row names angle rows inside the sinogram: k0 in [0, K), and the second angle
// row k0 + 1 < K unless the row wraps (k0 = K - 1, second row = row 0 mirrored).
__host__ __device__ inline bool row_geom_valid(const RowGeom& g, int K)
{
    return g.k0 >= 0 && g.k0 < K && (g.wrap == 0 ? g.k0 + 1 < K : (g.wrap == 1 && g.k0 == K - 1));
}

// Transposed resampling table.  Sinogram rows are taken kRsRows at a time; an entry is one
// linogram row whose resampling reads rows of the group: code = 2 (q N + i) + mirrored
// (1: the row-0 read past the last angle, detector mirrored), w[r] = its weight into group
// row r (w0 for its angle row k0, w1 for k0 + 1, 0 for the others).
constexpr int kRsRows = 4;
struct ReaderEntry {
    int code;
    float w[kRsRows];
};

// Fast Radon transform, per sinogram row k: the line class q holding theta_k, the two
// linogram rows i0, i0 + 1 around its slope with weights (1 - t, t), the path length per
// row `scale` = sqrt(1 + sigma^2), and per row the stored column of detector bin m,
// c = a m + b in 32.32 fixed point.
struct RadonRow {
    int q, i0;
    float t, scale;
    long long a_fx[2], b_fx[2];
};
}  // namespace fbp

struct fbp_plan_s {
    int N, K, M, batch;
    int n, n1, n2;          // log2 N, Hough stages in pass 1 and pass 2
    int chunk;              // slices processed per kernel sequence
    int device;
    fbp_iir_coeffs coeffs;
    fbp::IirParams iir;
    fbp::RowGeom* d_geom;   // [4][N]
    float2* d_trig;         // [K] (cos, sin) for the direct comparator
    int* d_readers;         // transposed-resampling table, per group of kRsRows sinogram
                            // rows: [groups + 1] CSR offsets into d_reader_ent
    fbp::ReaderEntry* d_reader_ent;
    int n_reader_ent;       // entries of d_reader_ent
    float2* d_hough_w;      // [4][N]: ((1 - ft), ft) / sqrt(1 + sigma^2), Hough-space data
    fbp::RadonRow* d_radon; // [K]: the fast Radon transform's resampling
    float* d_sirt;          // SIRT tables of one slice, made on first use: R^-1 [4][N][2N],
                            // then C^-1 [N][N]
    int* d_status;          // device status word
    // workspace
    void* ws;
    size_t ws_bytes;
    int ws_owned;
    size_t off_filt, off_g, off_stage_sino[2], off_stage_img[2];
    // adjoint workspace (allocated on first use): per chunk slice two linogram-sized
    // buffers and one sinogram-sized buffer
    void* adj_ws;
    size_t adj_bytes;
    // host-API pipeline
    cudaStream_t st_h2d, st_comp, st_d2h;
    cudaEvent_t ev_start, ev_h2d[2], ev_comp[2], ev_free[2], ev_done;
    // measurement hooks
    long long launches[FBP_KERNEL_COUNT];
    int prof_on;
    struct Timed { int kernel; cudaEvent_t a, b; };
    std::vector<Timed> prof_pending;
    std::vector<cudaEvent_t> prof_pool;
    double prof_ms[FBP_KERNEL_COUNT];
};

namespace fbp {

// Kernel launchers (each returns cudaGetLastError() after the launch).
// out_pitch >= M: output rows are out_pitch floats apart, the M samples centred in each
// with (out_pitch - M) / 2 zeros before them and the rest after (guard bins).
// in_tab (device array, optional): slice s of the input is in_tab[s] instead of in + s K M.
cudaError_t launch_iir(const fbp_plan_s* p, const float* in, float* out, int rows,
                       int out_pitch, cudaStream_t st, const float* const* in_tab = nullptr);
cudaError_t launch_resample(const fbp_plan_s* p, const float* filt, float* lin, int count,
                            cudaStream_t st);
cudaError_t launch_pass1(const fbp_plan_s* p, const float* src, bool from_lin, float* g,
                         int count, cudaStream_t st);
// Second pass: horizontal == false launches the v quarters (stores F_v- + F_v+),
// horizontal == true the h quarters (adds F_h- + F_h+); the v launch must come first.
// img_tab (device array, optional): slice s of the image is img_tab[s] instead of img + s N N.
cudaError_t launch_pass2(const fbp_plan_s* p, const float* g, float* img, int count,
                         bool horizontal, cudaStream_t st, float* const* img_tab = nullptr);
cudaError_t launch_fir(const fbp_plan_s* p, const float* in, float* out, int rows,
                       cudaStream_t st);
// Adjoints: image gradient [count][N][N] -> linogram gradient [count][4][N][2N] (scratch:
// another [count][4][N][2N] buffer), and linogram gradient -> filtered-sinogram gradient
// [count][K][M] (zeroed, then scattered into).
// resid_b / resid_w (optional): write the SIRT residual (resid_b - A f) * resid_w instead
// of A f, resid_b [count][4][N][2N], resid_w one slice's [4][N][2N].
cudaError_t launch_fht_adjoint(const fbp_plan_s* p, const float* img_grad, float* lin_grad,
                               float* scratch, int count, cudaStream_t st,
                               const float* resid_b = nullptr, const float* resid_w = nullptr);
cudaError_t launch_resample_adjoint(const fbp_plan_s* p, const float* lin_grad, float* filt_grad,
                                    int count, cudaStream_t st);
cudaError_t launch_direct_bp(const fbp_plan_s* p, const float* filt, float* img, int count,
                             cudaStream_t st);
// Algebraic reconstruction (sirt.cu): Hough-space data of a sinogram [count][K][M] ->
// [count][4][N][2N]; f = f + lam * cinv * t elementwise, cinv one slice's [per_slice] array
// shared by all count slices (per_slice a multiple of 4); fill and reciprocal (0 where not
// positive).
cudaError_t launch_hough_data(const fbp_plan_s* p, const float* sino, float* lin, int count,
                              cudaStream_t st);
cudaError_t launch_sirt_update(float* f, const float* t, const float* cinv, float lam,
                               size_t per_slice, int count, cudaStream_t st);
cudaError_t launch_fill(float* x, float v, size_t n, cudaStream_t st);
// Fast Radon transform: dyadic line sums [count][4][N][2N] -> sinogram [count][K][M].
cudaError_t launch_radon(const fbp_plan_s* p, const float* lin, float* sino, int count,
                         cudaStream_t st);
cudaError_t launch_recip(float* x, size_t n, cudaStream_t st);

// The fused pipeline keeps its filtered sinogram with kGuard zero bins on both sides of
// every row, so resampling reads bins -kGuard .. M+kGuard-1 without range checks.
constexpr int kGuard = 2;
inline int filt_pitch(const fbp_plan_s* p) { return p->M + 2 * kGuard; }

// Plan internals shared by the entry points (fbp_api.cu) and the ragged volume (volume.cu).
int default_chunk(const fbp_plan_s* p);
void layout_workspace(fbp_plan_s* p, int chunk);
fbp_status ensure_workspace(fbp_plan_s* p);
// The fused pipeline over cnt consecutive slices of one chunk on stream st: filter ->
// (resample + pass 1) -> (pass 2 + sum).  sino_tab / img_tab (device arrays, optional)
// give the slices' own sinogram / image buffers instead of sino + s K M / img + s N N.
cudaError_t reconstruct_chunk(fbp_plan_s* p, const float* sino, float* img, int cnt,
                              cudaStream_t st, const float* const* sino_tab = nullptr,
                              float* const* img_tab = nullptr);

inline size_t lin_floats(const fbp_plan_s* p) { return (size_t)4 * p->N * 2 * p->N; }
inline size_t sino_floats(const fbp_plan_s* p) { return (size_t)p->K * p->M; }
inline size_t img_floats(const fbp_plan_s* p) { return (size_t)p->N * p->N; }

}  // namespace fbp
