// Ragged volumes: one call reconstructs slices of different sizes (N, K, M), each slice in
// its own caller buffers.
//
// Every kernel of the pipeline is specialised at compile time for its size class (Hough
// stages per pass, filter modes), and each N has its own fitted filter, so slices are
// grouped by (N, K, M) and every group runs the fused pipeline of its own plan, in chunks,
// on its own stream: groups of different sizes overlap on the GPU.  The kernels reach the
// slices through per-group device tables of the items' sinogram and image pointers, so no
// slice is copied.  The whole volume can be captured once into a CUDA graph and replayed.
// An autotuner picks, per group, the first-pass fusion depth and the slices per launch by
// timing them on the volume's own items (results are bit-identical for every choice).
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "fbp_internal.h"

struct fbp_volume_s {
    struct Group {
        int N, K, M;
        std::vector<int> items;          // indices into the caller's item array
        fbp_plan_s* plan = nullptr;
        const float** sino_tab = nullptr;   // device [items.size()]
        float** img_tab = nullptr;          // device [items.size()]
        cudaStream_t st = nullptr;
        cudaEvent_t done = nullptr;
    };
    int device = 0;
    int flags = 0;
    int order = 0;
    std::vector<Group> groups;
    void* d_tables = nullptr;
    cudaEvent_t fork = nullptr;
    cudaGraphExec_t graph = nullptr;
};

namespace {

bool aligned16(const void* ptr) { return ((uintptr_t)ptr & 15u) == 0; }

fbp_status cuda_status(cudaError_t e) { return e == cudaSuccess ? FBP_OK : FBP_ERR_CUDA; }

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

void destroy_volume(fbp_volume_s* v)
{
    if (!v) return;
    DeviceGuard g(v->device);
    cudaDeviceSynchronize();
    if (v->graph) cudaGraphExecDestroy(v->graph);
    for (auto& gr : v->groups) {
        if (gr.plan) fbp_plan_destroy(gr.plan);
        if (gr.st) cudaStreamDestroy(gr.st);
        if (gr.done) cudaEventDestroy(gr.done);
    }
    if (v->fork) cudaEventDestroy(v->fork);
    if (v->d_tables) cudaFree(v->d_tables);
    delete v;
}

// Every group's chunks on the group's stream, forked from and joined back into `st`.
cudaError_t enqueue(fbp_volume_s* v, cudaStream_t st)
{
    cudaError_t e = cudaEventRecord(v->fork, st);
    for (auto& gr : v->groups) {
        if (e != cudaSuccess) break;
        e = cudaStreamWaitEvent(gr.st, v->fork, 0);
        const int n = (int)gr.items.size();
        const int chunk = gr.plan->chunk;
        for (int c = 0; c < n && e == cudaSuccess; c += chunk) {
            const int cnt = n - c < chunk ? n - c : chunk;
            e = fbp::reconstruct_chunk(gr.plan, nullptr, nullptr, cnt, gr.st, gr.sino_tab + c,
                                       gr.img_tab + c);
        }
        if (e == cudaSuccess) e = cudaEventRecord(gr.done, gr.st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, gr.done, 0);
    }
    return e;
}

fbp_status ensure_all_workspaces(fbp_volume_s* v)
{
    for (auto& gr : v->groups) {
        const fbp_status s = fbp::ensure_workspace(gr.plan);
        if (s != FBP_OK) return s;
    }
    return FBP_OK;
}

// Re-lays a group's plan for `chunk` slices per launch, dropping an owned workspace that
// no longer fits (the next run allocates it again).
void set_group_chunk(fbp_plan_s* p, int chunk)
{
    const size_t old_bytes = p->ws_bytes;
    fbp::layout_workspace(p, chunk);
    if (p->ws && p->ws_owned && p->ws_bytes > old_bytes) {
        cudaFree(p->ws);
        p->ws = nullptr;
        p->ws_owned = 0;
    }
}

fbp_status make_plan(const fbp_volume_s* v, const fbp_volume_s::Group& gr, int fuse_k,
                     fbp_plan_s** out)
{
    fbp_iir_coeffs c;
    fbp_status s = fbp_default_coeffs(gr.N, v->order, &c);
    if (s != FBP_OK) return s;
    return fbp_plan(out, gr.N, gr.K, gr.M, (int)gr.items.size(), &c, fuse_k);
}

}  // namespace

extern "C" {

fbp_status fbp_volume_create(fbp_volume_t* out, const fbp_item* items, int count, int order,
                             int flags)
{
    if (!out) return FBP_ERR_INVALID_ARG;
    *out = nullptr;
    if (!items || count < 1 || (flags & ~FBP_VOLUME_GRAPH) != 0) return FBP_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i) {
        const fbp_item& it = items[i];
        if (!it.d_sino || !it.d_img) return FBP_ERR_INVALID_ARG;
        if (!aligned16(it.d_sino) || !aligned16(it.d_img)) return FBP_ERR_MISALIGNED;
        if (it.N < 2 || it.N > 4096 || (it.N & (it.N - 1)) != 0) return FBP_ERR_UNSUPPORTED;
        if (it.K < 2 || it.M < 2) return FBP_ERR_INVALID_ARG;
    }
    fbp_volume_s* v = new (std::nothrow) fbp_volume_s();
    if (!v) return FBP_ERR_OOM;
    v->flags = flags;
    v->order = order;
    if (cudaGetDevice(&v->device) != cudaSuccess) { delete v; return FBP_ERR_CUDA; }

    // group by shape, in order of first appearance
    std::map<std::tuple<int, int, int>, int> index;
    for (int i = 0; i < count; ++i) {
        const auto key = std::make_tuple(items[i].N, items[i].K, items[i].M);
        auto it = index.find(key);
        if (it == index.end()) {
            it = index.emplace(key, (int)v->groups.size()).first;
            v->groups.emplace_back();
            v->groups.back().N = items[i].N;
            v->groups.back().K = items[i].K;
            v->groups.back().M = items[i].M;
        }
        v->groups[it->second].items.push_back(i);
    }

    fbp_status st = FBP_OK;
    for (auto& gr : v->groups) {
        st = make_plan(v, gr, 0, &gr.plan);
        if (st != FBP_OK) break;
    }
    // pointer tables, laid out group after group
    std::vector<const void*> host(2 * (size_t)count);
    if (st == FBP_OK) {
        cudaError_t e = cudaMalloc(&v->d_tables, host.size() * sizeof(void*));
        if (e != cudaSuccess) st = FBP_ERR_OOM;
    }
    if (st == FBP_OK) {
        size_t off = 0;
        for (auto& gr : v->groups) {
            const size_t n = gr.items.size();
            void** base = static_cast<void**>(v->d_tables);
            gr.sino_tab = static_cast<const float**>(static_cast<void*>(base + off));
            gr.img_tab = static_cast<float**>(static_cast<void*>(base + count + off));
            for (size_t j = 0; j < n; ++j) {
                host[off + j] = items[gr.items[j]].d_sino;
                host[count + off + j] = items[gr.items[j]].d_img;
            }
            off += n;
        }
        cudaError_t e = cudaMemcpy(v->d_tables, host.data(), host.size() * sizeof(void*),
                                   cudaMemcpyHostToDevice);
        for (auto& gr : v->groups) {
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&gr.st, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&gr.done, cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&v->fork, cudaEventDisableTiming);
        st = cuda_status(e);
    }
    if (st == FBP_OK) st = ensure_all_workspaces(v);
    if (st != FBP_OK) {
        destroy_volume(v);
        return st;
    }
    *out = v;
    return FBP_OK;
}

fbp_status fbp_volume_run(fbp_volume_t v, void* stream)
{
    if (!v) return FBP_ERR_INVALID_ARG;
    DeviceGuard g(v->device);
    if (!g.ok) return FBP_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    fbp_status s = ensure_all_workspaces(v);
    if (s != FBP_OK) return s;
    if (!(v->flags & FBP_VOLUME_GRAPH)) return cuda_status(enqueue(v, st));

    if (st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread)
        return FBP_ERR_INVALID_ARG;                     // capture needs a created stream
    if (!v->graph) {
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t e1 = enqueue(v, st);
            e = cudaStreamEndCapture(st, &graph);
            if (e1 != cudaSuccess) e = e1;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&v->graph, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            v->graph = nullptr;
            cudaGetLastError();
            return FBP_ERR_CUDA;
        }
    }
    return cuda_status(cudaGraphLaunch(v->graph, st));
}

fbp_status fbp_volume_tune(fbp_volume_t v, void* stream, int* fuse_k_out, int* chunk_out)
{
    if (!v) return FBP_ERR_INVALID_ARG;
    DeviceGuard g(v->device);
    if (!g.ok) return FBP_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    fbp_status s = cuda_status(e);
    for (size_t gi = 0; gi < v->groups.size() && s == FBP_OK; ++gi) {
        auto& gr = v->groups[gi];
        int n = 0;
        while ((1 << n) < gr.N) ++n;
        const int size = (int)gr.items.size();
        float best = -1.0f;
        int best_k = gr.plan->n1, best_c = gr.plan->chunk;
        // fusion depths the passes support: n <= 6 runs one pass of all n stages; larger
        // sizes split n = k + (n - k) with 2 <= k <= 6 and n - k <= 6
        for (int k = 1; k <= 6 && s == FBP_OK; ++k) {
            if (n <= 6 ? k != n : (k < 2 || n - k > 6)) continue;
            fbp_plan_s* p = nullptr;
            s = make_plan(v, gr, k, &p);
            if (s != FBP_OK) break;
            for (int c = 1; c <= 16 && c <= size && s == FBP_OK; c *= 2) {
                set_group_chunk(p, c);
                s = fbp::ensure_workspace(p);
                if (s != FBP_OK) break;
                float ms = 0.0f;
                for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {   // warm-up + 2 timed
                    if (rep == 1) e = cudaEventRecord(a, st);
                    for (int c0 = 0; c0 < size && e == cudaSuccess; c0 += c)
                        e = fbp::reconstruct_chunk(p, nullptr, nullptr, size - c0 < c ? size - c0 : c,
                                                   st, gr.sino_tab + c0, gr.img_tab + c0);
                }
                if (e == cudaSuccess) e = cudaEventRecord(b, st);
                if (e == cudaSuccess) e = cudaEventSynchronize(b);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
                s = cuda_status(e);
                if (s == FBP_OK && (best < 0.0f || ms < best)) {
                    best = ms;
                    best_k = k;
                    best_c = c;
                }
            }
            fbp_plan_destroy(p);
        }
        if (s != FBP_OK) break;
        if (best_k != gr.plan->n1) {
            fbp_plan_s* p = nullptr;
            s = make_plan(v, gr, best_k, &p);
            if (s != FBP_OK) break;
            fbp_plan_destroy(gr.plan);
            gr.plan = p;
        }
        set_group_chunk(gr.plan, best_c);
        if (fuse_k_out) fuse_k_out[gi] = best_k;
        if (chunk_out) chunk_out[gi] = best_c;
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (s == FBP_OK) s = ensure_all_workspaces(v);
    if (v->graph) {                                      // re-capture with the new plans
        cudaGraphExecDestroy(v->graph);
        v->graph = nullptr;
    }
    return s;
}

fbp_status fbp_volume_info(fbp_volume_t v, int* groups, size_t* workspace_bytes)
{
    if (!v) return FBP_ERR_INVALID_ARG;
    if (groups) *groups = (int)v->groups.size();
    if (workspace_bytes) {
        size_t total = 0;
        for (const auto& gr : v->groups) total += gr.plan->ws_bytes;
        *workspace_bytes = total;
    }
    return FBP_OK;
}

fbp_status fbp_volume_group(fbp_volume_t v, int group, int* N, int* K, int* M, int* items,
                            int* fuse_k, int* chunk)
{
    if (!v || group < 0 || group >= (int)v->groups.size()) return FBP_ERR_INVALID_ARG;
    const auto& gr = v->groups[group];
    if (N) *N = gr.N;
    if (K) *K = gr.K;
    if (M) *M = gr.M;
    if (items) *items = (int)gr.items.size();
    if (fuse_k) *fuse_k = gr.plan->n1;
    if (chunk) *chunk = gr.plan->chunk;
    return FBP_OK;
}

fbp_status fbp_volume_destroy(fbp_volume_t v)
{
    destroy_volume(v);
    return FBP_OK;
}

}  // extern "C"
