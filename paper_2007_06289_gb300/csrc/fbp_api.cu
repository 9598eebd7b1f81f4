// C ABI of libfbp: plans, geometry tables, workspace and the entry points of include/fbp.h.
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <complex>
#include <new>
#include <vector>

#include "fbp_internal.h"

namespace fbp {
cudaError_t prepare_fht_kernels();
cudaError_t prepare_iir_kernels();
cudaError_t prepare_direct_kernels();
cudaError_t prepare_adjoint_kernels();
}

namespace {

struct TableEntry {
    int N;
    int order;
    double b[FBP_MAX_ORDER];
    double a[FBP_MAX_ORDER];
};

const TableEntry kTable[] = {
#include "iir_table.inc"
};

constexpr int kDefaultOrder = 3;
constexpr size_t kAlign = 256;
constexpr size_t kChunkSlices = 16;                 // default slices per kernel sequence
constexpr size_t kChunkBytes = (size_t)4 << 30;     // cap on G per chunk
constexpr int kHostChunk = 2;                       // slices per staged copy of the host path
constexpr size_t kMaxChunk = 4096;

size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }
bool aligned16(const void* ptr) { return ((uintptr_t)ptr & 15u) == 0; }

fbp_status cuda_status(cudaError_t e) { return e == cudaSuccess ? FBP_OK : FBP_ERR_CUDA; }

// Switches to the plan's device for the lifetime of the guard.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard()
    {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Stability by the step-down (Schur-Cohn) recursion: all reflection coefficients |k| < 1.
bool stable(const double* a, int q)
{
    std::vector<double> c(a, a + q);
    for (int m = q; m >= 1; --m) {
        const double k = c[m - 1];
        if (!(fabs(k) < 1.0)) return false;
        std::vector<double> nc(m - 1);
        for (int j = 0; j < m - 1; ++j) nc[j] = (c[j] - k * c[m - 2 - j]) / (1.0 - k * k);
        c.swap(nc);
    }
    return true;
}

using cplx = std::complex<double>;

// Roots of the monic z^q + a[0] z^(q-1) + ... + a[q-1] (Aberth-Ehrlich iteration, then
// Newton polishing), q <= 8.
std::vector<cplx> poly_roots(const double* a, int q)
{
    std::vector<cplx> z(q);
    if (q == 0) return z;
    auto eval = [&](cplx x, cplx& dp) {
        cplx p = 1.0;
        dp = 0.0;
        for (int k = 0; k < q; ++k) {
            dp = dp * x + p;
            p = p * x + a[k];
        }
        return p;
    };
    double rad = 0.0;
    for (int k = 0; k < q; ++k) rad = fmax(rad, pow(fabs(a[k]), 1.0 / (k + 1)));
    rad = fmax(rad, 0.5);
    for (int i = 0; i < q; ++i) z[i] = std::polar(rad, 2.0 * M_PI * i / q + 0.4);
    for (int it = 0; it < 1000; ++it) {
        double worst = 0.0;
        for (int i = 0; i < q; ++i) {
            cplx dp;
            const cplx p = eval(z[i], dp);
            if (p == 0.0) continue;
            const cplx w = p / dp;
            cplx s = 0.0;
            for (int j = 0; j < q; ++j)
                if (j != i) s += 1.0 / (z[i] - z[j]);
            const cplx stepv = w / (1.0 - w * s);
            z[i] -= stepv;
            worst = fmax(worst, std::abs(stepv) / fmax(1.0, std::abs(z[i])));
        }
        if (worst < 1e-16) break;
    }
    for (int i = 0; i < q; ++i)
        for (int it = 0; it < 3; ++it) {
            cplx dp;
            const cplx p = eval(z[i], dp);
            if (std::abs(dp) > 0.0) z[i] -= p / dp;
        }
    return z;
}

// Parallel form of the causal filter B(w)/A(w), w = z^-1 (Eq. 9):
//   B(w)/A(w) = D(w) + sum_j r_j / (1 - p_j w),  p_j the roots of z^q + a_1 z^(q-1) + ...,
// D the polynomial part (present when mb > q).  Fills the kernel parameters and checks the
// realisation against the direct-form impulse response in float64.
fbp_status build_iir_params(fbp_plan_s* p)
{
    fbp::IirParams& prm = p->iir;
    memset(&prm, 0, sizeof(prm));
    // Split each row over wpr warps so that a lane holds at most kIirLmax samples; the
    // per-lane length L is odd (conflict-free strided shared-memory access).
    int wpr = 1;
    while (32 * wpr * fbp::kIirLmax < p->M) ++wpr;
    int L = (p->M + 32 * wpr - 1) / (32 * wpr);
    if ((L & 1) == 0) ++L;
    // The kernel has a fully unrolled variant for L = kIirLmax: take it when the lanes it
    // leaves idle (filtering zero padding) cost at most an eighth of the row.
    if ((long long)(32 * wpr * fbp::kIirLmax - p->M) * 8 <= p->M) L = fbp::kIirLmax;
    prm.L = L;
    prm.wpr = wpr;

    int q = p->coeffs.q;
    const int mb0 = p->coeffs.mb;
    while (q > 0 && p->coeffs.a[q - 1] == 0.0) --q;       // trailing zero coefficients
    const double* a = p->coeffs.a;
    const double* b = p->coeffs.b;

    // A DC-free numerator (B(1) = 0, as for the fitted ramp filters) factors as
    // B(w) = (1 - w) B'(w); the kernel then drives the modes with the first difference of
    // the input and realises B'/A.  Otherwise B/A is realised on the input itself.
    double bsum = 0.0, babs = 0.0;
    for (int k = 0; k < mb0; ++k) { bsum += b[k]; babs += fabs(b[k]); }
    std::vector<double> num(b, b + mb0);
    prm.diff = 0;
    if (mb0 >= 2 && fabs(bsum) <= 1e-12 * babs) {
        prm.diff = 1;
        num.assign(mb0 - 1, 0.0);
        double acc = 0.0;
        for (int k = 0; k < mb0 - 1; ++k) { acc += b[k]; num[k] = acc; }
    }
    const int mb = (int)num.size();

    // polynomial part and proper remainder (long division in powers of w)
    std::vector<double> rem(num), D;
    if (mb - 1 >= q) {
        if (q == 0) {
            D = rem;
            rem.assign(1, 0.0);
        } else {
            D.assign(mb - q, 0.0);
            for (int deg = mb - 1; deg >= q; --deg) {
                const double c = rem[deg] / a[q - 1];          // a_q is the w^q coefficient
                D[deg - q] = c;
                rem[deg - q] -= c;                             // w^0 coefficient of A is 1
                for (int k = 1; k <= q; ++k) rem[deg - q + k] -= c * a[k - 1];
            }
            rem.resize(q);
        }
    }
    if ((int)D.size() > fbp::kMaxOrder) return FBP_ERR_UNSUPPORTED;
    prm.nd = (int)D.size();
    for (int k = 0; k < prm.nd; ++k) prm.d[k] = (float)D[k];

    const std::vector<cplx> pole = poly_roots(a, q);
    for (int i = 0; i < q; ++i) {
        if (!(std::abs(pole[i]) < 1.0)) return FBP_ERR_INVALID_ARG;     // unstable
        for (int j = 0; j < i; ++j)
            if (std::abs(pole[i] - pole[j]) < 1e-7) return FBP_ERR_UNSUPPORTED;   // repeated
    }
    auto Bp = [&](cplx w) {
        cplx s = 0.0;
        for (int k = (int)rem.size() - 1; k >= 0; --k) s = s * w + rem[k];
        return s;
    };
    std::vector<cplx> res(q);
    for (int j = 0; j < q; ++j) {
        cplx den = 1.0;
        for (int i = 0; i < q; ++i)
            if (i != j) den *= 1.0 - pole[i] / pole[j];
        res[j] = Bp(1.0 / pole[j]) / den;
    }

    // impulse-response check of the parallel form against the recursion in float64
    {
        const int T = 96;
        std::vector<double> h(T, 0.0);
        double scale = 0.0;
        for (int n = 0; n < T; ++n) {
            double v = n < mb0 ? b[n] : 0.0;
            for (int k = 1; k <= q; ++k)
                if (n - k >= 0) v -= a[k - 1] * h[n - k];
            h[n] = v;
            scale = fmax(scale, fabs(v));
        }
        double err = 0.0;
        double gprev = 0.0;
        for (int n = 0; n < T; ++n) {
            cplx g = n < prm.nd ? D[n] : 0.0;
            for (int j = 0; j < q; ++j) g += res[j] * std::pow(pole[j], n);
            const double gn = g.real();
            err = fmax(err, fabs((prm.diff ? gn - gprev : gn) - h[n]));
            gprev = gn;
        }
        if (!(err <= 1e-9 * fmax(scale, 1e-300))) return FBP_ERR_UNSUPPORTED;
    }

    // real modes, and one representative (Im p > 0) per conjugate pair with doubled residue
    for (int j = 0; j < q; ++j) {
        const cplx pj = pole[j];
        const bool real = fabs(pj.imag()) <= 1e-12 * fmax(1.0, std::abs(pj));
        cplx carry = std::pow(pj, L);
        if (real) {
            const int m = prm.jr++;
            prm.rp[m] = (float)pj.real();
            prm.rr[m] = (float)res[j].real();
            double c = carry.real();
            for (int d = 0; d < fbp::kScanSteps; ++d, c *= c) prm.rpow[d][m] = (float)c;
            prm.rwarp[m] = (float)std::pow(pj, 32 * L).real();
        } else if (pj.imag() > 0.0) {
            const int m = prm.jc++;
            prm.cpr[m] = (float)pj.real();
            prm.cpi[m] = (float)pj.imag();
            prm.crr[m] = (float)(2.0 * res[j].real());
            prm.cri[m] = (float)(2.0 * res[j].imag());
            for (int d = 0; d < fbp::kScanSteps; ++d, carry *= carry) {
                prm.cpowr[d][m] = (float)carry.real();
                prm.cpowi[d][m] = (float)carry.imag();
            }
            const cplx pw = std::pow(pj, 32 * L);
            prm.cwarpr[m] = (float)pw.real();
            prm.cwarpi[m] = (float)pw.imag();
        }
    }
    if (prm.jr + 2 * prm.jc != q) return FBP_ERR_UNSUPPORTED;     // unpaired complex root
    return FBP_OK;
}

long long to_fixed(double v) { return llround(ldexp(v, fbp::kFixBits)); }

// Per (quarter, row) sampling geometry, computed in float64 (Sec. 4.1-4.2, Eq. 14-15).
// Quarter order v-, v+, h-, h+; row i has slope sigma = i/(N-1).  Normal angle theta:
// atan(sigma), pi - atan(sigma), pi/2 - atan(sigma), pi/2 + atan(sigma).  For stored
// column c (intercept u = c, or N-1-c for the '+' quarters) the signed offset from the
// centre c0 is r = (c - c0 (1 + sigma)) / sqrt(1 + sigma^2), negated for h+.
std::vector<fbp::RowGeom> build_geometry(int N, int K, int M,
                                         std::vector<float2>* hough_w = nullptr)
{
    std::vector<fbp::RowGeom> g(4 * (size_t)N);
    if (hough_w) hough_w->assign(4 * (size_t)N, make_float2(0.0f, 0.0f));
    const double c0 = 0.5 * (N - 1);
    const double half = 0.5 * (M - 1);
    for (int q = 0; q < 4; ++q) {
        for (int i = 0; i < N; ++i) {
            const double s = (double)i / (N - 1);
            const double at = atan(s);
            double theta;
            switch (q) {
                case 0: theta = at; break;
                case 1: theta = M_PI - at; break;
                case 2: theta = 0.5 * M_PI - at; break;
                default: theta = 0.5 * M_PI + at; break;
            }
            double tk = theta * K / M_PI;
            double k0 = floor(tk);
            if (k0 > K - 1) k0 = K - 1;
            fbp::RowGeom& e = g[(size_t)q * N + i];
            e.k0 = (int)k0;
            const double ft = tk - k0;
            e.wrap = (e.k0 + 1 >= K) ? 1 : 0;
            double w = (1.0 / (N - 1)) / (1.0 + s * s);
            if (i == 0 || i == N - 1) w *= 0.5;
            e.w0 = (float)(w * (1.0 - ft));
            e.w1 = (float)(w * ft);
            const double inv = 1.0 / sqrt(1.0 + s * s);
            if (hough_w)        // angle weights over the path length per row, no w
                (*hough_w)[(size_t)q * N + i] = make_float2((float)((1.0 - ft) * inv), (float)(ft * inv));
            double A = inv, B = -c0 * (1.0 + s) * inv;
            if (q == 3) { A = -A; B = -B; }
            e.a_fx = to_fixed(A);
            e.b_fx = to_fixed(B + half);
        }
    }
    return g;
}

// Transposed-resampling table: per group of kRsRows sinogram rows, the linogram rows whose
// resampling reads any row of the group (Eq. 14-15: row (q, i) interpolates between angle
// rows k0 and k0 + 1 with weights w0 and w1, or, past the last angle, between k0 and row 0
// with the detector mirrored), each with its weight into every row of the group.  A row
// whose two angle rows fall in different groups appears in both.  Entries are in (q, i)
// order, mirrored reads after the direct ones of group 0.
struct ReaderTable {
    std::vector<int> ptr;
    std::vector<fbp::ReaderEntry> ent;
};

ReaderTable build_readers(const std::vector<fbp::RowGeom>& geo, int K)
{
    const int R = fbp::kRsRows;
    const int groups = (K + R - 1) / R;
    std::vector<std::vector<fbp::ReaderEntry>> per(groups);
    std::vector<fbp::ReaderEntry> mirrored;
    auto add = [&](int row, int code, float w) {
        std::vector<fbp::ReaderEntry>& v = per[row / R];
        if (v.empty() || v.back().code != code) {
            fbp::ReaderEntry e{code, {}};
            v.push_back(e);
        }
        v.back().w[row % R] += w;
    };
    for (size_t qi = 0; qi < geo.size(); ++qi) {
        const fbp::RowGeom& g = geo[qi];
        add(g.k0, (int)qi * 2, g.w0);
        if (!g.wrap) {
            add(g.k0 + 1, (int)qi * 2, g.w1);
        } else {
            fbp::ReaderEntry e{(int)qi * 2 + 1, {}};
            e.w[0] = g.w1;
            mirrored.push_back(e);
        }
    }
    per[0].insert(per[0].end(), mirrored.begin(), mirrored.end());
    ReaderTable t;
    t.ptr.resize(groups + 1);
    t.ptr[0] = 0;
    for (int gi = 0; gi < groups; ++gi) {
        t.ptr[gi + 1] = t.ptr[gi] + (int)per[gi].size();
        t.ent.insert(t.ent.end(), per[gi].begin(), per[gi].end());
    }
    return t;
}

// Fast Radon transform table (float64 geometry, then 32.32 fixed point): per sinogram row,
// the line class holding theta_k (v- up to pi/4, h- up to pi/2, h+ up to 3pi/4, v+ beyond;
// slope sigma = tan of the angle to the class's axis), the two linogram rows around
// sigma (N-1), and in each the stored column of detector bin m: the row's offset r is affine
// in the column, r(c) = r0 + dr c, so c = (m - (M-1)/2 - r0) / dr.
double class_angle(int q, double s)
{
    const double at = atan(s);
    switch (q) {
        case 0: return at;
        case 1: return M_PI - at;
        case 2: return 0.5 * M_PI - at;
        default: return 0.5 * M_PI + at;
    }
}

double class_offset(int q, double s, double c, int N)     // r of stored column c
{
    const double c0 = 0.5 * (N - 1);
    const double th = class_angle(q, s);
    const double u = (q == 0 || q == 2) ? c : (N - 1) - c;
    const double x = q < 2 ? u : 0.0, y = q < 2 ? 0.0 : u;
    return (x - c0) * cos(th) + (y - c0) * sin(th);
}

std::vector<fbp::RadonRow> build_radon(int N, int K, int M)
{
    std::vector<fbp::RadonRow> t(K);
    for (int k = 0; k < K; ++k) {
        const double th = k * M_PI / K;
        int q;
        double s;
        if (th <= M_PI / 4) { q = 0; s = tan(th); }
        else if (th <= M_PI / 2) { q = 2; s = tan(M_PI / 2 - th); }
        else if (th <= 3 * M_PI / 4) { q = 3; s = tan(th - M_PI / 2); }
        else { q = 1; s = tan(M_PI - th); }
        const double istar = s * (N - 1);
        int i0 = (int)floor(istar);
        if (i0 > N - 2) i0 = N - 2;
        if (i0 < 0) i0 = 0;
        fbp::RadonRow& e = t[k];
        e.q = q;
        e.i0 = i0;
        e.t = (float)(istar - i0);
        e.scale = (float)sqrt(1.0 + s * s);
        for (int j = 0; j < 2; ++j) {
            const double si = (double)(i0 + j) / (N - 1);
            const double r0 = class_offset(q, si, 0.0, N);
            const double dr = class_offset(q, si, 1.0, N) - r0;
            e.a_fx[j] = to_fixed(1.0 / dr);
            e.b_fx[j] = to_fixed((-0.5 * (M - 1) - r0) / dr);
        }
    }
    return t;
}

int ilog2(int v)
{
    int n = 0;
    while ((1 << n) < v) ++n;
    return n;
}

float* ws_ptr(const fbp_plan_s* p, size_t off) { return (float*)((char*)p->ws + off); }

cudaEvent_t prof_event(fbp_plan_s* p)
{
    if (!p->prof_pool.empty()) {
        cudaEvent_t e = p->prof_pool.back();
        p->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Issues one kernel launch `f` on stream st, counting it and, with profiling on, bracketing
// it with CUDA events on the same stream.
template <class F>
cudaError_t run(fbp_plan_s* p, int kernel, cudaStream_t st, F&& f)
{
    cudaEvent_t a = nullptr, b = nullptr;
    if (p->prof_on) {
        a = prof_event(p);
        b = prof_event(p);
        if (a && b) cudaEventRecord(a, st);
    }
    const cudaError_t e = f();
    if (a && b) {
        cudaEventRecord(b, st);
        p->prof_pending.push_back({kernel, a, b});
    } else {
        if (a) p->prof_pool.push_back(a);
        if (b) p->prof_pool.push_back(b);
    }
    if (e == cudaSuccess) ++p->launches[kernel];
    return e;
}

// Folds finished event pairs into the per-kernel totals.
cudaError_t prof_collect(fbp_plan_s* p)
{
    cudaError_t err = cudaSuccess;
    for (const fbp_plan_s::Timed& t : p->prof_pending) {
        float ms = 0.0f;
        cudaError_t e = cudaEventSynchronize(t.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t.a, t.b);
        if (e == cudaSuccess) p->prof_ms[t.kernel] += ms;
        else err = e;
        p->prof_pool.push_back(t.a);
        p->prof_pool.push_back(t.b);
    }
    p->prof_pending.clear();
    return err;
}

}  // namespace

namespace fbp {

// Slices per kernel sequence.  Larger chunks give every launch a larger grid (fewer
// partial waves, fewer dependent-launch gaps) at the price of a working set that no longer
// stays in L2; the kernels are not DRAM-bound, so the grid size wins (measured on GB300 at
// N = 2048, slices/s for 1, 2, 4, 8, 16 slices per launch: 5590, 6456, 7062, 7459, 7670).
int default_chunk(const fbp_plan_s* p)
{
    size_t chunk = kChunkSlices;
    const size_t g_bytes = fbp::lin_floats(p) * sizeof(float);
    if (chunk * g_bytes > kChunkBytes) chunk = kChunkBytes / g_bytes;
    if (chunk < 1) chunk = 1;
    if (chunk > (size_t)p->batch) chunk = p->batch;
    return (int)chunk;
}

// Workspace offsets for `chunk` slices per kernel sequence: filtered sinogram (guarded
// rows), first-pass buffer G, and two staging slots each for the host pipeline.
void layout_workspace(fbp_plan_s* p, int chunk)
{
    const size_t s_bytes = fbp::sino_floats(p) * sizeof(float);
    const size_t f_bytes = (size_t)p->K * fbp::filt_pitch(p) * sizeof(float);
    const size_t g_bytes = fbp::lin_floats(p) * sizeof(float);
    p->chunk = chunk;
    size_t off = 0;
    p->off_filt = off; off = align_up(off + chunk * f_bytes);
    p->off_g = off; off = align_up(off + chunk * g_bytes);
    for (int b = 0; b < 2; ++b) { p->off_stage_sino[b] = off; off = align_up(off + chunk * s_bytes); }
    for (int b = 0; b < 2; ++b) {
        p->off_stage_img[b] = off;
        off = align_up(off + chunk * fbp::img_floats(p) * sizeof(float));
    }
    p->ws_bytes = off;
}

fbp_status ensure_workspace(fbp_plan_s* p)
{
    if (p->ws) return FBP_OK;
    void* ws = nullptr;
    if (cudaMalloc(&ws, p->ws_bytes) != cudaSuccess) {
        cudaGetLastError();
        return FBP_ERR_OOM;
    }
    p->ws = ws;
    p->ws_owned = 1;
    return FBP_OK;
}

// One chunk of the fused pipeline: filter -> (resample + pass 1) -> (pass 2 + sum).
cudaError_t reconstruct_chunk(fbp_plan_s* p, const float* sino, float* img, int cnt,
                              cudaStream_t st, const float* const* sino_tab, float* const* img_tab)
{
    float* filt = ws_ptr(p, p->off_filt);
    float* g = ws_ptr(p, p->off_g);
    cudaError_t e = run(p, FBP_KERNEL_IIR, st,
                        [&] { return launch_iir(p, sino, filt, cnt * p->K, filt_pitch(p), st, sino_tab); });
    if (e == cudaSuccess)
        e = run(p, FBP_KERNEL_PASS1_RESAMPLE, st,
                [&] { return launch_pass1(p, filt, false, g, cnt, st); });
    if (e == cudaSuccess)
        e = run(p, FBP_KERNEL_PASS2, st,
                [&] { return launch_pass2(p, g, img, cnt, false, st, img_tab); });
    if (e == cudaSuccess && p->n2 > 0)
        e = run(p, FBP_KERNEL_PASS2_H, st,
                [&] { return launch_pass2(p, g, img, cnt, true, st, img_tab); });
    return e;
}

}  // namespace fbp

using fbp::default_chunk;
using fbp::ensure_workspace;
using fbp::layout_workspace;
using fbp::reconstruct_chunk;

extern "C" {

const char* fbp_status_str(fbp_status s)
{
    switch (s) {
        case FBP_OK: return "ok";
        case FBP_ERR_INVALID_ARG: return "invalid argument";
        case FBP_ERR_UNSUPPORTED: return "unsupported size or order";
        case FBP_ERR_MISALIGNED: return "pointer not 16-byte aligned";
        case FBP_ERR_OOM: return "out of memory";
        case FBP_ERR_CUDA: return "CUDA error";
        case FBP_ERR_TIMEOUT: return "bounded wait timed out";
        case FBP_ERR_INTERNAL: return "internal consistency check failed";
    }
    return "unknown status";
}

fbp_status fbp_default_coeffs(int N, int order, fbp_iir_coeffs* out)
{
    if (!out) return FBP_ERR_INVALID_ARG;
    if (order <= 0) order = kDefaultOrder;
    for (const TableEntry& t : kTable) {
        if (t.N == N && t.order == order) {
            memset(out, 0, sizeof(*out));
            out->mb = order;
            out->q = order;
            for (int k = 0; k < order; ++k) {
                out->b[k] = t.b[k];
                out->a[k] = t.a[k];
            }
            return FBP_OK;
        }
    }
    return FBP_ERR_UNSUPPORTED;
}

fbp_status fbp_plan(fbp_plan_t* out, int N, int K, int M, int batch,
                    const fbp_iir_coeffs* coeffs, int fuse_k)
{
    if (!out) return FBP_ERR_INVALID_ARG;
    *out = nullptr;
    if (N < 2 || N > 4096 || (N & (N - 1)) != 0) return FBP_ERR_UNSUPPORTED;
    if (K < 2 || M < 2 || M > 32 * fbp::kIirMaxWarps * fbp::kIirLmax || batch < 1)
        return FBP_ERR_INVALID_ARG;
    fbp_iir_coeffs c;
    if (coeffs) {
        c = *coeffs;
    } else {
        fbp_status st = fbp_default_coeffs(N, 0, &c);
        if (st != FBP_OK) return st;
    }
    if (c.mb < 1 || c.mb > FBP_MAX_ORDER || c.q < 0 || c.q > FBP_MAX_ORDER)
        return FBP_ERR_UNSUPPORTED;
    double ad[FBP_MAX_ORDER];
    for (int k = 0; k < c.mb; ++k)
        if (!isfinite(c.b[k])) return FBP_ERR_INVALID_ARG;
    for (int k = 0; k < c.q; ++k) {
        if (!isfinite(c.a[k])) return FBP_ERR_INVALID_ARG;
        ad[k] = c.a[k];
    }
    if (!stable(ad, c.q)) return FBP_ERR_INVALID_ARG;

    const int n = ilog2(N);
    int n1, n2;
    if (fuse_k == 0) {
        n1 = n <= 6 ? n : (n + 1) / 2;
    } else {
        if (fuse_k < 1 || fuse_k > 6) return FBP_ERR_UNSUPPORTED;
        n1 = fuse_k < n ? fuse_k : n;
    }
    n2 = n - n1;
    // a second pass needs first-pass blocks of at least 4 rows (its rows then fit the
    // 2N-float G rows with their 16-byte alignment shift)
    if (n2 > 6 || (n2 > 0 && n1 < 2)) return FBP_ERR_UNSUPPORTED;

    fbp_plan_s* p = new (std::nothrow) fbp_plan_s();
    if (!p) return FBP_ERR_OOM;
    p->N = N; p->K = K; p->M = M; p->batch = batch;
    p->n = n; p->n1 = n1; p->n2 = n2;
    p->coeffs = c;
    {
        const fbp_status fs = build_iir_params(p);
        if (fs != FBP_OK) { delete p; return fs; }
    }
    if (cudaGetDevice(&p->device) != cudaSuccess) { delete p; return FBP_ERR_CUDA; }

    layout_workspace(p, default_chunk(p));

    fbp_status st = FBP_OK;
    std::vector<float2> hough_w;
    std::vector<fbp::RowGeom> geo = build_geometry(N, K, M, &hough_w);
    std::vector<float2> trig(K);
    for (int k = 0; k < K; ++k) {
        const double th = k * M_PI / K;
        trig[k] = make_float2((float)cos(th), (float)sin(th));
    }
    const ReaderTable readers = build_readers(geo, K);
    p->n_reader_ent = (int)readers.ent.size();
    cudaError_t e = cudaMalloc(&p->d_geom, geo.size() * sizeof(fbp::RowGeom));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_trig, trig.size() * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_readers, readers.ptr.size() * sizeof(int));
    if (e == cudaSuccess)
        e = cudaMalloc(&p->d_reader_ent, readers.ent.size() * sizeof(fbp::ReaderEntry));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_hough_w, hough_w.size() * sizeof(float2));
    const std::vector<fbp::RadonRow> radon = build_radon(N, K, M);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_radon, radon.size() * sizeof(fbp::RadonRow));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_status, sizeof(int));
    if (e != cudaSuccess) st = FBP_ERR_OOM;
    if (st == FBP_OK) {
        e = cudaMemcpy(p->d_geom, geo.data(), geo.size() * sizeof(fbp::RowGeom), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(p->d_trig, trig.data(), trig.size() * sizeof(float2), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(p->d_readers, readers.ptr.data(), readers.ptr.size() * sizeof(int),
                           cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(p->d_reader_ent, readers.ent.data(),
                           readers.ent.size() * sizeof(fbp::ReaderEntry), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(p->d_hough_w, hough_w.data(), hough_w.size() * sizeof(float2),
                           cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(p->d_radon, radon.data(), radon.size() * sizeof(fbp::RadonRow),
                           cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, sizeof(int));
        if (e == cudaSuccess) e = fbp::prepare_fht_kernels();
        if (e == cudaSuccess) e = fbp::prepare_iir_kernels();
        if (e == cudaSuccess) e = fbp::prepare_direct_kernels();
        if (e == cudaSuccess) e = fbp::prepare_adjoint_kernels();
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->st_h2d, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->st_comp, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->st_d2h, cudaStreamNonBlocking);
        const unsigned ef = cudaEventDisableTiming;
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_start, ef);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_done, ef);
        for (int b = 0; b < 2; ++b) {
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_h2d[b], ef);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_comp[b], ef);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_free[b], ef);
        }
        if (e != cudaSuccess) st = FBP_ERR_CUDA;
    }
    if (st != FBP_OK) {
        cudaGetLastError();
        fbp_plan_destroy(p);
        return st;
    }
    *out = p;
    return FBP_OK;
}

fbp_status fbp_plan_destroy(fbp_plan_t p)
{
    if (!p) return FBP_OK;
    DeviceGuard g(p->device);
    cudaDeviceSynchronize();
    if (p->ws_owned && p->ws) cudaFree(p->ws);
    if (p->adj_ws) cudaFree(p->adj_ws);
    if (p->d_geom) cudaFree(p->d_geom);
    if (p->d_trig) cudaFree(p->d_trig);
    if (p->d_readers) cudaFree(p->d_readers);
    if (p->d_reader_ent) cudaFree(p->d_reader_ent);
    if (p->d_hough_w) cudaFree(p->d_hough_w);
    if (p->d_radon) cudaFree(p->d_radon);
    if (p->d_sirt) cudaFree(p->d_sirt);
    if (p->d_status) cudaFree(p->d_status);
    cudaStream_t ss[3] = {p->st_h2d, p->st_comp, p->st_d2h};
    for (cudaStream_t s : ss)
        if (s) cudaStreamDestroy(s);
    cudaEvent_t es[2] = {p->ev_start, p->ev_done};
    for (cudaEvent_t ev : es)
        if (ev) cudaEventDestroy(ev);
    for (const fbp_plan_s::Timed& t : p->prof_pending) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    for (cudaEvent_t ev : p->prof_pool) cudaEventDestroy(ev);
    for (int b = 0; b < 2; ++b) {
        if (p->ev_h2d[b]) cudaEventDestroy(p->ev_h2d[b]);
        if (p->ev_comp[b]) cudaEventDestroy(p->ev_comp[b]);
        if (p->ev_free[b]) cudaEventDestroy(p->ev_free[b]);
    }
    cudaGetLastError();
    delete p;
    return FBP_OK;
}

size_t fbp_workspace_bytes(fbp_plan_t p) { return p ? p->ws_bytes : 0; }

fbp_status fbp_set_chunk(fbp_plan_t p, int chunk)
{
    if (!p || p->ws) return FBP_ERR_INVALID_ARG;
    if (chunk == 0) chunk = default_chunk(p);
    if (chunk < 1 || chunk > p->batch || (size_t)chunk > kMaxChunk) return FBP_ERR_INVALID_ARG;
    layout_workspace(p, chunk);
    return FBP_OK;
}

fbp_status fbp_set_workspace(fbp_plan_t p, void* d_ws, size_t bytes)
{
    if (!p) return FBP_ERR_INVALID_ARG;
    if (d_ws && bytes < p->ws_bytes) return FBP_ERR_INVALID_ARG;
    if (d_ws && !aligned16(d_ws)) return FBP_ERR_MISALIGNED;
    if (p->ws_owned && p->ws) {
        DeviceGuard g(p->device);
        cudaDeviceSynchronize();
        cudaFree(p->ws);
    }
    p->ws = d_ws;
    p->ws_owned = 0;
    return FBP_OK;
}

fbp_status fbp_plan_info(fbp_plan_t p, int* N, int* K, int* M, int* batch, int* fuse_k,
                         int* chunk)
{
    if (!p) return FBP_ERR_INVALID_ARG;
    if (N) *N = p->N;
    if (K) *K = p->K;
    if (M) *M = p->M;
    if (batch) *batch = p->batch;
    if (fuse_k) *fuse_k = p->n1;
    if (chunk) *chunk = p->chunk;
    return FBP_OK;
}

fbp_status fbp_filter_iir(fbp_plan_t p, const float* d_sino, float* d_filt, void* stream)
{
    if (!p || !d_sino || !d_filt) return FBP_ERR_INVALID_ARG;
    if (!aligned16(d_sino) || !aligned16(d_filt)) return FBP_ERR_MISALIGNED;
    DeviceGuard g(p->device);
    if (!g.ok) return FBP_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    return cuda_status(run(p, FBP_KERNEL_IIR, st, [&] {
        return fbp::launch_iir(p, d_sino, d_filt, p->batch * p->K, p->M, st);
    }));
}

fbp_status fbp_filter_fir(fbp_plan_t p, const float* d_sino, float* d_filt, void* stream)
{
    if (!p || !d_sino || !d_filt || d_sino == d_filt) return FBP_ERR_INVALID_ARG;
    if (!aligned16(d_sino) || !aligned16(d_filt)) return FBP_ERR_MISALIGNED;
    DeviceGuard g(p->device);
    if (!g.ok) return FBP_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    return cuda_status(run(p, FBP_KERNEL_FIR, st, [&] {
        return fbp::launch_fir(p, d_sino, d_filt, p->batch * p->K, st);
    }));
}

fbp_status fbp_resample_st(fbp_plan_t p, const float* d_filt, float* d_lin, void* stream)
{
    if (!p || !d_filt || !d_lin) return FBP_ERR_INVALID_ARG;
    if (!aligned16(d_filt) || !aligned16(d_lin)) return FBP_ERR_MISALIGNED;
    DeviceGuard g(p->device);
    if (!g.ok) return FBP_ERR_CUDA;
    for (int c = 0; c < p->batch; c += p->chunk) {
        const int cnt = p->batch - c < p->chunk ? p->batch - c : p->chunk;
        cudaStream_t st = (cudaStream_t)stream;
        cudaError_t e = run(p, FBP_KERNEL_RESAMPLE, st, [&] {
            return fbp::launch_resample(p, d_filt + (size_t)c * fbp::sino_floats(p),
                                        d_lin + (size_t)c * fbp::lin_floats(p), cnt, st);
        });
        if (e != cudaSuccess) return FBP_ERR_CUDA;
    }
    return FBP_OK;
}

}  // extern "C"

namespace {

// Back projection of cnt linograms (pass 1 from the linogram, pass 2 with the quarter sum)
// through the workspace's first-pass buffer.
cudaError_t backproject_lin_chunk(fbp_plan_s* p, const float* lin, float* img, int cnt,
                                  cudaStream_t st)
{
    float* gbuf = ws_ptr(p, p->off_g);
    cudaError_t e = run(p, FBP_KERNEL_PASS1_LINOGRAM, st,
                        [&] { return fbp::launch_pass1(p, lin, true, gbuf, cnt, st); });
    if (e == cudaSuccess)
        e = run(p, FBP_KERNEL_PASS2, st, [&] { return fbp::launch_pass2(p, gbuf, img, cnt, false, st); });
    if (e == cudaSuccess && p->n2 > 0)
        e = run(p, FBP_KERNEL_PASS2_H, st, [&] { return fbp::launch_pass2(p, gbuf, img, cnt, true, st); });
    return e;
}

}  // namespace

extern "C" {

fbp_status fbp_fht_backproject(fbp_plan_t p, const float* d_lin, float* d_img, void* stream)
{
    if (!p || !d_lin || !d_img) return FBP_ERR_INVALID_ARG;
    if (!aligned16(d_lin) || !aligned16(d_img)) return FBP_ERR_MISALIGNED;
    DeviceGuard g(p->device);
    if (!g.ok) return FBP_ERR_CUDA;
    fbp_status s = ensure_workspace(p);
    if (s != FBP_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    for (int c = 0; c < p->batch; c += p->chunk) {
        const int cnt = p->batch - c < p->chunk ? p->batch - c : p->chunk;
        const cudaError_t e = backproject_lin_chunk(p, d_lin + (size_t)c * fbp::lin_floats(p),
                                                    d_img + (size_t)c * fbp::img_floats(p), cnt, st);
        if (e != cudaSuccess) return FBP_ERR_CUDA;
    }
    return FBP_OK;
}

fbp_status fbp_reconstruct(fbp_plan_t p, const float* d_sino, float* d_img, void* stream)
{
    if (!p || !d_sino || !d_img) return FBP_ERR_INVALID_ARG;
    if (!aligned16(d_sino) || !aligned16(d_img)) return FBP_ERR_MISALIGNED;
    DeviceGuard g(p->device);
    if (!g.ok) return FBP_ERR_CUDA;
    fbp_status s = ensure_workspace(p);
    if (s != FBP_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    for (int c = 0; c < p->batch; c += p->chunk) {
        const int cnt = p->batch - c < p->chunk ? p->batch - c : p->chunk;
        cudaError_t e = reconstruct_chunk(p, d_sino + (size_t)c * fbp::sino_floats(p),
                                          d_img + (size_t)c * fbp::img_floats(p), cnt, st);
        if (e != cudaSuccess) return FBP_ERR_CUDA;
    }
    return FBP_OK;
}

fbp_status fbp_reconstruct_host(fbp_plan_t p, const float* h_sino, float* h_img, int count,
                                void* stream)
{
    if (!p || !h_sino || !h_img || count < 1) return FBP_ERR_INVALID_ARG;
    DeviceGuard g(p->device);
    if (!g.ok) return FBP_ERR_CUDA;
    fbp_status s = ensure_workspace(p);
    if (s != FBP_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t sf = fbp::sino_floats(p), imf = fbp::img_floats(p);
    cudaError_t e = cudaEventRecord(p->ev_start, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->st_h2d, p->ev_start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->st_comp, p->ev_start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->st_d2h, p->ev_start, 0);
    // Small staged chunks keep the pipeline's fill and drain short: the copies, not the
    // kernels, bound this path.
    const int hc = p->chunk < kHostChunk ? p->chunk : kHostChunk;
    int ci = 0;
    for (int c = 0; c < count && e == cudaSuccess; c += hc, ++ci) {
        const int b = ci & 1;
        const int cnt = count - c < hc ? count - c : hc;
        float* dsino = ws_ptr(p, p->off_stage_sino[b]);
        float* dimg = ws_ptr(p, p->off_stage_img[b]);
        if (ci >= 2) e = cudaStreamWaitEvent(p->st_h2d, p->ev_comp[b], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dsino, h_sino + (size_t)c * sf, (size_t)cnt * sf * sizeof(float),
                                cudaMemcpyHostToDevice, p->st_h2d);
        if (e == cudaSuccess) e = cudaEventRecord(p->ev_h2d[b], p->st_h2d);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p->st_comp, p->ev_h2d[b], 0);
        if (e == cudaSuccess && ci >= 2) e = cudaStreamWaitEvent(p->st_comp, p->ev_free[b], 0);
        if (e == cudaSuccess) e = reconstruct_chunk(p, dsino, dimg, cnt, p->st_comp);
        if (e == cudaSuccess) e = cudaEventRecord(p->ev_comp[b], p->st_comp);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p->st_d2h, p->ev_comp[b], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_img + (size_t)c * imf, dimg, (size_t)cnt * imf * sizeof(float),
                                cudaMemcpyDeviceToHost, p->st_d2h);
        if (e == cudaSuccess) e = cudaEventRecord(p->ev_free[b], p->st_d2h);
    }
    if (e == cudaSuccess) e = cudaEventRecord(p->ev_done, p->st_d2h);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, p->ev_done, 0);
    return cuda_status(e);
}

// ------------------------------------------------------------------ adjoints
namespace {

fbp_status ensure_adjoint_workspace(fbp_plan_s* p)
{
    const size_t lin = fbp::lin_floats(p) * sizeof(float);
    const size_t sino = fbp::sino_floats(p) * sizeof(float);
    const size_t need = (size_t)p->chunk * (2 * lin + sino);
    if (p->adj_ws && p->adj_bytes >= need) return FBP_OK;
    if (p->adj_ws) {
        cudaDeviceSynchronize();
        cudaFree(p->adj_ws);
        p->adj_ws = nullptr;
        p->adj_bytes = 0;
    }
    if (cudaMalloc(&p->adj_ws, need) != cudaSuccess) {
        cudaGetLastError();
        p->adj_ws = nullptr;
        return FBP_ERR_OOM;
    }
    p->adj_bytes = need;
    return FBP_OK;
}

float* adj_lin(const fbp_plan_s* p, int which)
{
    return (float*)p->adj_ws + (size_t)which * p->chunk * fbp::lin_floats(p);
}

}  // namespace

fbp_status fbp_fht_backproject_adjoint(fbp_plan_t p, const float* d_img_grad, float* d_lin_grad,
                                       void* stream)
{
    if (!p || !d_img_grad || !d_lin_grad) return FBP_ERR_INVALID_ARG;
    if (!aligned16(d_img_grad) || !aligned16(d_lin_grad)) return FBP_ERR_MISALIGNED;
    DeviceGuard g(p->device);
    if (!g.ok) return FBP_ERR_CUDA;
    fbp_status s = ensure_adjoint_workspace(p);
    if (s != FBP_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    for (int c = 0; c < p->batch; c += p->chunk) {
        const int cnt = p->batch - c < p->chunk ? p->batch - c : p->chunk;
        const cudaError_t e = fbp::launch_fht_adjoint(
            p, d_img_grad + (size_t)c * fbp::img_floats(p),
            d_lin_grad + (size_t)c * fbp::lin_floats(p), adj_lin(p, 1), cnt, st);
        if (e != cudaSuccess) return FBP_ERR_CUDA;
    }
    return FBP_OK;
}

fbp_status fbp_hough_project(fbp_plan_t p, const float* d_img, float* d_lin, void* stream)
{
    return fbp_fht_backproject_adjoint(p, d_img, d_lin, stream);
}

fbp_status fbp_resample_st_adjoint(fbp_plan_t p, const float* d_lin_grad, float* d_filt_grad,
                                   void* stream)
{
    if (!p || !d_lin_grad || !d_filt_grad) return FBP_ERR_INVALID_ARG;
    if (!aligned16(d_lin_grad) || !aligned16(d_filt_grad)) return FBP_ERR_MISALIGNED;
    DeviceGuard g(p->device);
    if (!g.ok) return FBP_ERR_CUDA;
    for (int c = 0; c < p->batch; c += p->chunk) {      // grid z is the chunk's slice count
        const int cnt = p->batch - c < p->chunk ? p->batch - c : p->chunk;
        const cudaError_t e = fbp::launch_resample_adjoint(
            p, d_lin_grad + (size_t)c * fbp::lin_floats(p),
            d_filt_grad + (size_t)c * fbp::sino_floats(p), cnt, (cudaStream_t)stream);
        if (e != cudaSuccess) return FBP_ERR_CUDA;
    }
    return FBP_OK;
}

fbp_status fbp_reconstruct_adjoint(fbp_plan_t p, const float* d_img_grad, float* d_sino_grad,
                                   void* stream)
{
    if (!p || !d_img_grad || !d_sino_grad) return FBP_ERR_INVALID_ARG;
    if (!aligned16(d_img_grad) || !aligned16(d_sino_grad)) return FBP_ERR_MISALIGNED;
    DeviceGuard g(p->device);
    if (!g.ok) return FBP_ERR_CUDA;
    fbp_status s = ensure_adjoint_workspace(p);
    if (s != FBP_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    float* lin = adj_lin(p, 0);
    float* scratch = adj_lin(p, 1);
    float* pbar = adj_lin(p, 2);
    for (int c = 0; c < p->batch; c += p->chunk) {
        const int cnt = p->batch - c < p->chunk ? p->batch - c : p->chunk;
        cudaError_t e = fbp::launch_fht_adjoint(p, d_img_grad + (size_t)c * fbp::img_floats(p),
                                                lin, scratch, cnt, st);
        if (e == cudaSuccess) e = fbp::launch_resample_adjoint(p, lin, pbar, cnt, st);
        // the filter is its own adjoint (Eq. 12-13: causal + anticausal is symmetric)
        if (e == cudaSuccess)
            e = fbp::launch_iir(p, pbar, d_sino_grad + (size_t)c * fbp::sino_floats(p),
                                cnt * p->K, p->M, st);
        if (e != cudaSuccess) return FBP_ERR_CUDA;
    }
    return FBP_OK;
}

// ------------------------------------------------------------------ algebraic reconstruction
fbp_status fbp_hough_data(fbp_plan_t p, const float* d_sino, float* d_lin, void* stream)
{
    if (!p || !d_sino || !d_lin) return FBP_ERR_INVALID_ARG;
    if (!aligned16(d_sino) || !aligned16(d_lin)) return FBP_ERR_MISALIGNED;
    DeviceGuard g(p->device);
    if (!g.ok) return FBP_ERR_CUDA;
    for (int c = 0; c < p->batch; c += p->chunk) {      // grid z is the chunk's slice count
        const int cnt = p->batch - c < p->chunk ? p->batch - c : p->chunk;
        const cudaError_t e = fbp::launch_hough_data(p, d_sino + (size_t)c * fbp::sino_floats(p),
                                                     d_lin + (size_t)c * fbp::lin_floats(p), cnt,
                                                     (cudaStream_t)stream);
        if (e != cudaSuccess) return FBP_ERR_CUDA;
    }
    return FBP_OK;
}

fbp_status fbp_radon(fbp_plan_t p, const float* d_img, float* d_sino, void* stream)
{
    if (!p || !d_img || !d_sino) return FBP_ERR_INVALID_ARG;
    if (!aligned16(d_img) || !aligned16(d_sino)) return FBP_ERR_MISALIGNED;
    DeviceGuard g(p->device);
    if (!g.ok) return FBP_ERR_CUDA;
    fbp_status s = ensure_adjoint_workspace(p);
    if (s != FBP_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    float* lin = adj_lin(p, 0);
    for (int c = 0; c < p->batch; c += p->chunk) {
        const int cnt = p->batch - c < p->chunk ? p->batch - c : p->chunk;
        cudaError_t e = fbp::launch_fht_adjoint(p, d_img + (size_t)c * fbp::img_floats(p), lin,
                                                adj_lin(p, 1), cnt, st);   // line sums, Eq. 17
        if (e == cudaSuccess)
            e = fbp::launch_radon(p, lin, d_sino + (size_t)c * fbp::sino_floats(p), cnt, st);
        if (e != cudaSuccess) return FBP_ERR_CUDA;
    }
    return FBP_OK;
}

namespace {

// R^-1 = 1 / (A 1) and C^-1 = 1 / (A^T 1) of one slice (0 where those vanish), made once per
// plan on `st` with the operators themselves.
fbp_status ensure_sirt_tables(fbp_plan_s* p, cudaStream_t st)
{
    if (p->d_sirt) return FBP_OK;
    const size_t lf = fbp::lin_floats(p), imf = fbp::img_floats(p);
    float* t = nullptr;
    if (cudaMalloc(&t, (lf + imf) * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return FBP_ERR_OOM;
    }
    float* ones_img = ws_ptr(p, p->off_stage_img[0]);
    float* ones_lin = adj_lin(p, 0);
    cudaError_t e = fbp::launch_fill(ones_img, 1.0f, imf, st);
    if (e == cudaSuccess) e = fbp::launch_fht_adjoint(p, ones_img, t, adj_lin(p, 1), 1, st);
    if (e == cudaSuccess) e = fbp::launch_recip(t, lf, st);
    if (e == cudaSuccess) e = fbp::launch_fill(ones_lin, 1.0f, lf, st);
    if (e == cudaSuccess) e = backproject_lin_chunk(p, ones_lin, t + lf, 1, st);
    if (e == cudaSuccess) e = fbp::launch_recip(t + lf, imf, st);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(st);
        cudaFree(t);
        return FBP_ERR_CUDA;
    }
    p->d_sirt = t;
    return FBP_OK;
}

}  // namespace

fbp_status fbp_sirt(fbp_plan_t p, const float* d_lin_data, float* d_img, int iters, float lambda,
                    void* stream)
{
    if (!p || !d_lin_data || !d_img || iters < 0) return FBP_ERR_INVALID_ARG;
    if (!(lambda > 0.0f && lambda < 2.0f)) return FBP_ERR_INVALID_ARG;
    if (!aligned16(d_lin_data) || !aligned16(d_img)) return FBP_ERR_MISALIGNED;
    DeviceGuard g(p->device);
    if (!g.ok) return FBP_ERR_CUDA;
    fbp_status s = ensure_workspace(p);
    if (s == FBP_OK) s = ensure_adjoint_workspace(p);
    cudaStream_t st = (cudaStream_t)stream;
    if (s == FBP_OK) s = ensure_sirt_tables(p, st);
    if (s != FBP_OK) return s;
    const size_t lf = fbp::lin_floats(p), imf = fbp::img_floats(p);
    const float* rinv = p->d_sirt;
    const float* cinv = p->d_sirt + lf;
    float* ax = adj_lin(p, 0);
    float* scratch = adj_lin(p, 1);
    float* atr = ws_ptr(p, p->off_stage_img[0]);
    for (int c = 0; c < p->batch; c += p->chunk) {
        const int cnt = p->batch - c < p->chunk ? p->batch - c : p->chunk;
        const float* b = d_lin_data + (size_t)c * lf;
        float* f = d_img + (size_t)c * imf;
        for (int it = 0; it < iters; ++it) {
            // r = (b - A f) R^-1, formed as the projection's last launch writes A f
            cudaError_t e = fbp::launch_fht_adjoint(p, f, ax, scratch, cnt, st, b, rinv);
            if (e == cudaSuccess) e = backproject_lin_chunk(p, ax, atr, cnt, st);     // A^T r
            if (e == cudaSuccess) e = fbp::launch_sirt_update(f, atr, cinv, lambda, imf, cnt, st);
            if (e != cudaSuccess) return FBP_ERR_CUDA;
        }
    }
    return FBP_OK;
}

fbp_status fbp_direct_reconstruct(fbp_plan_t p, const float* d_sino, float* d_img, void* stream)
{
    if (!p || !d_sino || !d_img) return FBP_ERR_INVALID_ARG;
    if (!aligned16(d_sino) || !aligned16(d_img)) return FBP_ERR_MISALIGNED;
    DeviceGuard g(p->device);
    if (!g.ok) return FBP_ERR_CUDA;
    fbp_status s = ensure_workspace(p);
    if (s != FBP_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    float* filt = ws_ptr(p, p->off_filt);
    for (int c = 0; c < p->batch; c += p->chunk) {
        const int cnt = p->batch - c < p->chunk ? p->batch - c : p->chunk;
        cudaError_t e = run(p, FBP_KERNEL_FIR, st, [&] {
            return fbp::launch_fir(p, d_sino + (size_t)c * fbp::sino_floats(p), filt, cnt * p->K, st);
        });
        if (e == cudaSuccess)
            e = run(p, FBP_KERNEL_DIRECT_BP, st, [&] {
                return fbp::launch_direct_bp(p, filt, d_img + (size_t)c * fbp::img_floats(p), cnt, st);
            });
        if (e != cudaSuccess) return FBP_ERR_CUDA;
    }
    return FBP_OK;
}

fbp_status fbp_profile_enable(fbp_plan_t p, int enable)
{
    if (!p) return FBP_ERR_INVALID_ARG;
    p->prof_on = enable ? 1 : 0;
    return FBP_OK;
}

fbp_status fbp_profile_reset(fbp_plan_t p)
{
    if (!p) return FBP_ERR_INVALID_ARG;
    DeviceGuard g(p->device);
    if (!g.ok) return FBP_ERR_CUDA;
    const cudaError_t e = prof_collect(p);
    for (int k = 0; k < FBP_KERNEL_COUNT; ++k) {
        p->prof_ms[k] = 0.0;
        p->launches[k] = 0;
    }
    return cuda_status(e);
}

fbp_status fbp_profile_read(fbp_plan_t p, int kernel, double* total_ms, long long* launches)
{
    if (!p || kernel < 0 || kernel >= FBP_KERNEL_COUNT) return FBP_ERR_INVALID_ARG;
    DeviceGuard g(p->device);
    if (!g.ok) return FBP_ERR_CUDA;
    const cudaError_t e = prof_collect(p);
    if (total_ms) *total_ms = p->prof_ms[kernel];
    if (launches) *launches = p->launches[kernel];
    return cuda_status(e);
}

fbp_status fbp_last_device_error(fbp_plan_t p)
{
    if (!p) return FBP_ERR_INVALID_ARG;
    DeviceGuard g(p->device);
    if (!g.ok) return FBP_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return FBP_ERR_CUDA;
    int v = 0;
    if (cudaMemcpy(&v, p->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return FBP_ERR_CUDA;
    if (v != 0 && cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess) return FBP_ERR_CUDA;
    return (fbp_status)v;
}

#ifdef FBP_BOUNDS_CHECK
#include "../../include/fbp_check.h"

fbp_status fbp_check_set_row_angle(fbp_plan_t p, int q, int i, int k0)
{
    if (!p || q < 0 || q >= 4 || i < 0 || i >= p->N) return FBP_ERR_INVALID_ARG;
    DeviceGuard g(p->device);
    if (!g.ok) return FBP_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return FBP_ERR_CUDA;
    fbp::RowGeom* row = p->d_geom + (size_t)q * p->N + i;
    return cudaMemcpy(&row->k0, &k0, sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess
               ? FBP_OK : FBP_ERR_CUDA;
}
#endif

}  // extern "C"
