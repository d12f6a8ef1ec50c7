// stb_batch.cu -- C ABI of the batched mixed-precision assembly: workspace
// layout, per-problem set-up, the persistent launch, and the tile autotuner.
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "stb_assemble.h"

namespace stb {

// Workspace: [status 256 B][descriptors][counter 256 B][problem 0][problem 1]...
struct BatchLayout {
    BatchDesc *descs;
    unsigned long long *counter;
    std::vector<AssemblyLayout> items;
    size_t bytes;
};

static stb_status batch_check(const stb_batch_item *items, int32_t n) {
    if (!items || n < 1) return fail(STB_ERR_INVALID_ARG, "need items and n >= 1");
    for (int i = 0; i < n; ++i) {
        const stb_batch_item &it = items[i];
        if (!it.mesh || !it.V) return fail(STB_ERR_INVALID_ARG, "item %d: mesh and V must be given", i);
        stb_status st = check_assembly_params(&it.params);
        if (st) return st;
        if (it.params.precision != STB_PREC_MIXED || it.params.storage != STB_STORE_F32)
            return fail(STB_ERR_INVALID_ARG,
                        "item %d: batches need STB_PREC_MIXED and STB_STORE_F32", i);
        if (it.mesh->m.n_tris > 65535)
            return fail(STB_ERR_INVALID_ARG, "item %d: dense assembly supports E <= 65535", i);
        if (it.params.quad_regular * it.params.quad_regular > 256)
            return fail(STB_ERR_INVALID_ARG, "item %d: quad_regular must be <= 16", i);
    }
    return STB_OK;
}

static BatchLayout batch_layout(const stb_batch_item *items, int n, void *ws, size_t cap) {
    BatchLayout B;
    char *base = static_cast<char *>(ws);
    size_t off = 256;
    B.descs = reinterpret_cast<BatchDesc *>(base ? base + off : nullptr);
    off += batch_desc_bytes(n);
    B.counter = reinterpret_cast<unsigned long long *>(base ? base + off : nullptr);
    off += 256;
    for (int i = 0; i < n; ++i) {
        const size_t need =
            align256(assembly_layout(items[i].mesh->m, items[i].params, nullptr, 0).bytes);
        void *sub = base ? base + off : nullptr;
        B.items.push_back(assembly_layout(items[i].mesh->m, items[i].params, sub,
                                          base && cap > off ? cap - off : 0));
        off += need;
    }
    B.bytes = off;
    return B;
}

static stb_status cu(cudaError_t e, const char *what) {
    return e == cudaSuccess ? STB_OK : cuda_fail(e, what);
}

// The problems' arrays as the batched launcher takes them.
struct BatchArgs {
    std::vector<const Mesh *> meshes;
    std::vector<stb_params> params;
    std::vector<float *> V, K;
};

// The problems' arrays as the batched launcher takes them.
static BatchArgs batch_args(const stb_batch_item *items, int n) {
    BatchArgs A;
    for (int i = 0; i < n; ++i) {
        A.meshes.push_back(&items[i].mesh->m);
        A.params.push_back(items[i].params);
        A.V.push_back(items[i].V);
        A.K.push_back(items[i].K);
    }
    return A;
}

// Set-up of every problem (tables, geometry, pair classification) and the
// descriptors for work items of `tile` columns.
static stb_status batch_prepare(const BatchLayout &B, const BatchArgs &A, int n, int tile,
                                void *ws, cudaStream_t s) {
    int32_t *status = status_word(ws);
    for (int i = 0; i < n; ++i) {
        stb_status st = prepare_mixed(*A.meshes[i], A.params[i], B.items[i], status, s);
        if (st) return st;
    }
    return upload_batch(A.meshes.data(), A.params.data(), B.items.data(), A.V.data(), A.K.data(),
                        n, B.descs, tile, s);
}

static stb_status batch_launch(const BatchLayout &B, const BatchArgs &A, int n, int tile,
                               int stride, cudaStream_t s) {
    return launch_batch(A.meshes.data(), A.params.data(), B.items.data(), A.V.data(), A.K.data(),
                        n, B.descs, B.counter, tile, stride, s);
}

// Tuned tiles per (device, batch shape): the shape is the number of problems
// and the binary orders of magnitude of the pair-step work and of the
// largest step count.
using Shape = std::tuple<int, int, int, int>;
static std::mutex g_tune_mu;
static std::map<Shape, int> g_tuned;

static Shape batch_shape(const stb_batch_item *items, int n) {
    double work = 0.0;
    int max_steps = 1, dev = 0;
    cudaGetDevice(&dev);
    for (int i = 0; i < n; ++i) {
        const double E = (double)items[i].mesh->m.n_tris;
        work += E * E * items[i].params.n_steps;
        max_steps = std::max(max_steps, items[i].params.n_steps);
    }
    return Shape(dev, n, (int)std::lround(std::log2(std::max(1.0, work))),
                 (int)std::lround(std::log2((double)max_steps)));
}

}  // namespace stb

using namespace stb;

extern "C" stb_status stb_batch_workspace_size(const stb_batch_item *items, int32_t n,
                                               size_t *bytes) {
    if (!bytes) return fail(STB_ERR_INVALID_ARG, "bytes must be given");
    stb_status st = batch_check(items, n);
    if (st) return st;
    *bytes = align256(batch_layout(items, n, nullptr, 0).bytes);
    return STB_OK;
}

static int resolve_tile(const stb_batch_item *items, int n, int tile) {
    if (tile != 0) return tile;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto f = g_tuned.find(batch_shape(items, n));
    return f != g_tuned.end() ? f->second : 128;
}

static stb_status batch_enter(const stb_batch_item *items, int32_t n, int32_t tile, void *ws,
                              size_t ws_bytes, BatchLayout &B) {
    stb_status st = batch_check(items, n);
    if (st) return st;
    if (tile != 0 && tile != 128 && tile != 256)
        return fail(STB_ERR_INVALID_ARG, "tile must be 0, 128 or 256");
    B = batch_layout(items, n, ws, ws_bytes);
    return check_workspace(ws, ws_bytes, B.bytes);
}

extern "C" stb_status stb_batch_prepare(const stb_batch_item *items, int32_t n, int32_t tile,
                                        void *ws, size_t ws_bytes, stb_stream stream) {
    BatchLayout B;
    stb_status st = batch_enter(items, n, tile, ws, ws_bytes, B);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    STB_CUDA(cudaMemsetAsync(ws, 0, 256, s));
    return batch_prepare(B, batch_args(items, n), n, resolve_tile(items, n, tile), ws, s);
}

extern "C" stb_status stb_batch_launch(const stb_batch_item *items, int32_t n, int32_t tile,
                                       void *ws, size_t ws_bytes, stb_stream stream) {
    BatchLayout B;
    stb_status st = batch_enter(items, n, tile, ws, ws_bytes, B);
    if (st) return st;
    return batch_launch(B, batch_args(items, n), n, resolve_tile(items, n, tile), 1,
                        (cudaStream_t)stream);
}

extern "C" stb_status stb_batch_assemble(const stb_batch_item *items, int32_t n, int32_t tile,
                                         void *ws, size_t ws_bytes, stb_stream stream) {
    stb_status st = stb_batch_prepare(items, n, tile, ws, ws_bytes, stream);
    if (st) return st;
    return stb_batch_launch(items, n, tile, ws, ws_bytes, stream);
}

extern "C" stb_status stb_batch_tune(const stb_batch_item *items, int32_t n, void *ws,
                                     size_t ws_bytes, stb_stream stream, int32_t *tile) {
    if (!tile) return fail(STB_ERR_INVALID_ARG, "tile must be given");
    BatchLayout B;
    stb_status st = batch_enter(items, n, 128, ws, ws_bytes, B);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    STB_CUDA(cudaMemsetAsync(ws, 0, 256, s));
    const BatchArgs A = batch_args(items, n);
    if ((st = batch_prepare(B, A, n, 128, ws, s))) return st;
    cudaEvent_t e0, e1;
    STB_CUDA(cudaEventCreate(&e0));
    STB_CUDA(cudaEventCreate(&e1));
    const int cand[2] = {128, 256};
    int best = 128;
    float best_ms = 0.f;
    for (int c = 0; c < 2 && !st; ++c) {
        st = upload_batch(A.meshes.data(), A.params.data(), B.items.data(), A.V.data(),
                          A.K.data(), n, B.descs, cand[c], s);
        if (!st) st = batch_launch(B, A, n, cand[c], 16, s);  // warm-up of this instantiation
        if (!st) st = cu(cudaEventRecord(e0, s), "cudaEventRecord");
        if (!st) st = batch_launch(B, A, n, cand[c], 16, s);
        if (!st) st = cu(cudaEventRecord(e1, s), "cudaEventRecord");
        if (!st) st = cu(cudaEventSynchronize(e1), "cudaEventSynchronize");
        float ms = 0.f;
        if (!st) st = cu(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
        if (!st && (c == 0 || ms < best_ms)) {
            best_ms = ms;
            best = cand[c];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[batch_shape(items, n)] = best;
    }
    *tile = best;
    return stb_workspace_status(ws, stream);
}
