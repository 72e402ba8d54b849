// group2d.cu -- many 2D grids advanced together: one persistent launch per time
// step moves every unfinished member grid on by one step of the fused TM
// scheme (the k_tm2d tile body, Sec. 2.3 update per cell), whatever the
// members' sizes, masses, couplings and fields.
//
// Work items are (member, x strip, y chunk) tiles of all members, taken from an
// atomic queue by a grid of resident blocks.  The block finishing the last tile
// of a member in a launch advances that member's step counter; the last block
// of the launch rewinds the queue.  A member's buffer roles alternate with
// period two, so each member carries the kernel parameters of both parities
// and a tile picks the set its member's step count selects.  Nothing waits on
// another block: completion is counted with atomics only.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "kernels_tm2d.cuh"
#include "kernels_tm2d_x2.cuh"

namespace axp {

bool tm2d_eligible(const axp_grid *g);
template <typename T>
fused::Params<T> tm2d_params(axp_grid *g, int chunk);

namespace {

struct GItem {
    int32_t member, bx, by, pad_;
};

struct GDev {
    const fused::Params<float> *params;  // [max_grids][2]
    int64_t *done, *steps;               // per member
    int32_t *cnt, *nblk;                 // tiles finished in this launch; tiles per step
    const GItem *items;
    int32_t nitems;
    int32_t *counter, *finished;
};

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct GLayout {
    size_t params, done, steps, cnt, nblk, items, counter, total;
};

GLayout glayout(int32_t max_grids, int32_t max_tiles)
{
    GLayout L;
    size_t off = 0;
    L.params = off;
    off += align_up(sizeof(fused::Params<float>) * 2 * (size_t)max_grids);
    L.done = off;
    off += align_up(sizeof(int64_t) * max_grids);
    L.steps = off;
    off += align_up(sizeof(int64_t) * max_grids);
    L.cnt = off;
    off += align_up(sizeof(int32_t) * max_grids);
    L.nblk = off;
    off += align_up(sizeof(int32_t) * max_grids);
    L.items = off;
    off += align_up(sizeof(GItem) * (size_t)max_tiles);
    L.counter = off;
    off += align_up(2 * sizeof(int32_t));
    L.total = off;
    return L;
}

// Blocks of kGroupThreads threads.  A member of even width takes tiles of the
// two-column form (2 kGroupThreads columns per tile); a member of odd width the
// one-column tile body (kGroupThreads columns).
constexpr int kGroupThreads = tm2d_x2::NTX;
constexpr int kVxPair = 2 * kGroupThreads - tm2d_x2::HL - tm2d_x2::HR;  // written columns per tile
constexpr int kVxOne = kGroupThreads - tm2d::HL - tm2d::HR;
constexpr size_t kGroupStage = tm2d_x2::stage_bytes(kGroupThreads);
static_assert(tm2d::stage_bytes<float>(kGroupThreads) <= kGroupStage, "one staging buffer serves both forms");

__host__ __device__ inline int group_vx(int64_t nx) { return nx % 2 == 0 ? kVxPair : kVxOne; }

__global__ void __launch_bounds__(kGroupThreads, 2) k_tm2d_group(GDev D)
{
    // the published rows of either form
    constexpr size_t kRowsOne = sizeof(float) * 2 * tm2d::NROWS * tm2d::RS;
    constexpr size_t kRowsPair = sizeof(float2) * 2 * tm2d_x2::NROWS * tm2d_x2::RS;
    __shared__ __align__(16) unsigned char rows_raw[kRowsOne > kRowsPair ? kRowsOne : kRowsPair];
    extern __shared__ __align__(16) unsigned char group_dyn[];
    __shared__ fused::Params<float> sP;
    __shared__ int s_item;
    __shared__ long long s_done;
    constexpr int kWords = sizeof(fused::Params<float>) / sizeof(int);
    static_assert(sizeof(fused::Params<float>) % sizeof(int) == 0, "Params copied as words");
    for (;;) {
        if (threadIdx.x == 0) {
            const int it = atomicAdd(D.counter, 1);
            s_item = it;
            // the member's step count is stable while any of its tiles is unfinished
            s_done = it < D.nitems ? (long long)__ldcg(D.done + D.items[it].member) : 0;
        }
        __syncthreads();
        const int it = s_item;
        if (it >= D.nitems) break;
        const GItem I = D.items[it];
        const int64_t done = s_done;
        if (done < __ldcg(D.steps + I.member)) {
            const int *src = (const int *)(D.params + 2 * (size_t)I.member + (done & 1));
            for (int k = threadIdx.x; k < kWords; k += kGroupThreads) ((int *)&sP)[k] = src[k];
            __syncthreads();
            if (sP.n[0] % 2 == 0)
                tm2d_x2::tile(sP, I.bx, I.by,
                              *reinterpret_cast<float2(*)[2][tm2d_x2::NROWS][tm2d_x2::RS]>(rows_raw),
                              reinterpret_cast<float2 *>(group_dyn));
            else
                tm2d::tile<float, true>(sP, I.bx, I.by, *reinterpret_cast<float(*)[2][tm2d::NROWS][tm2d::RS]>(rows_raw),
                                        reinterpret_cast<float *>(group_dyn));
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();  // this tile's stores before the count that publishes them
                if (atomicAdd(D.cnt + I.member, 1) == D.nblk[I.member] - 1) {
                    D.cnt[I.member] = 0;
                    D.done[I.member] = done + 1;
                }
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(D.finished, 1) == (int)gridDim.x - 1) {
            // every block has taken its last item: rewind the queue for the next launch
            *D.counter = 0;
            *D.finished = 0;
        }
    }
}

axp_status cuda_st(cudaError_t e)
{
    if (e == cudaSuccess) return AXP_OK;
    if (e == cudaErrorMemoryAllocation) return AXP_E_NOMEM;
    fprintf(stderr, "axp_group: CUDA error %s\n", cudaGetErrorString(e));
    return AXP_E_CUDA;
}

}  // namespace
}  // namespace axp

using namespace axp;

struct axp_group {
    int32_t max_grids, max_tiles;
    char *ws;
    cudaStream_t stream;
    GLayout L;
    GDev D;
    struct Member {
        axp_grid *g;
        int64_t steps;
        int32_t nblk, active;
    };
    std::vector<Member> members;
    int32_t chunk;  // y planes per tile
    bool dirty;
    int grid_blocks;
    int64_t launches;
    bool use_graph;
    cudaGraphExec_t graph;
    int64_t graph_steps;
};

namespace {

void drop_graph(axp_group *G)
{
    if (G->graph) cudaGraphExecDestroy(G->graph);
    G->graph = nullptr;
    G->graph_steps = -1;
}

int32_t tiles_of(const axp_grid *g, int32_t chunk)
{
    const int vx = group_vx(g->desc.n[0]);
    const int64_t strips = (g->desc.n[0] + vx - 1) / vx;
    const int64_t chunks = (g->desc.n[1] + chunk - 1) / chunk;
    return (int32_t)(strips * chunks);
}

axp_status rebuild(axp_group *G)
{
    std::vector<GItem> items;
    for (int m = 0; m < G->max_grids; m++) {
        const auto &M = G->members[m];
        if (!M.active) continue;
        const int vx = group_vx(M.g->desc.n[0]);
        const int strips = (int)((M.g->desc.n[0] + vx - 1) / vx);
        const int chunks = (int)((M.g->desc.n[1] + G->chunk - 1) / G->chunk);
        for (int by = 0; by < chunks; by++)
            for (int bx = 0; bx < strips; bx++) items.push_back({m, bx, by, 0});
    }
    if ((int64_t)items.size() > G->max_tiles) return AXP_E_NOMEM;
    cudaError_t e = cudaSuccess;
    if (!items.empty())
        e = cudaMemcpyAsync(G->ws + G->L.items, items.data(), items.size() * sizeof(GItem), cudaMemcpyHostToDevice,
                            G->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(G->stream);
    if (e != cudaSuccess) return cuda_st(e);
    G->D.nitems = (int32_t)items.size();
    G->dirty = false;
    return AXP_OK;
}

cudaError_t enqueue(axp_group *G, int64_t nsteps)
{
    const int grid = std::max(1, std::min(G->grid_blocks, G->D.nitems));
    for (int64_t s = 0; s < nsteps; s++) {
        k_tm2d_group<<<grid, kGroupThreads, kGroupStage, G->stream>>>(G->D);
        G->launches++;
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

axp_status axp_group_workspace_bytes(int32_t max_grids, int32_t max_tiles, size_t *bytes)
{
    if (!bytes || max_grids < 1 || max_tiles < 1) return AXP_E_INVAL;
    *bytes = glayout(max_grids, max_tiles).total;
    return AXP_OK;
}

axp_status axp_group_create(int32_t max_grids, int32_t max_tiles, void *dev_workspace, size_t bytes, void *cuda_stream,
                            axp_group **out)
{
    if (!out || !dev_workspace || max_grids < 1 || max_tiles < 1) return AXP_E_INVAL;
    if ((uintptr_t)dev_workspace % kAlign) return AXP_E_INVAL;
    *out = nullptr;
    const GLayout L = glayout(max_grids, max_tiles);
    if (bytes < L.total) return AXP_E_NOMEM;
    axp_group *G = new (std::nothrow) axp_group();
    if (!G) return AXP_E_NOMEM;
    G->max_grids = max_grids;
    G->max_tiles = max_tiles;
    G->ws = (char *)dev_workspace;
    G->stream = (cudaStream_t)cuda_stream;
    G->L = L;
    G->D.params = (const fused::Params<float> *)(G->ws + L.params);
    G->D.done = (int64_t *)(G->ws + L.done);
    G->D.steps = (int64_t *)(G->ws + L.steps);
    G->D.cnt = (int32_t *)(G->ws + L.cnt);
    G->D.nblk = (int32_t *)(G->ws + L.nblk);
    G->D.items = (const GItem *)(G->ws + L.items);
    G->D.nitems = 0;
    G->D.counter = (int32_t *)(G->ws + L.counter);
    G->D.finished = G->D.counter + 1;
    G->members.assign(max_grids, axp_group::Member{nullptr, 0, 0, 0});
    G->chunk = 64;
    G->dirty = true;
    G->launches = 0;
    G->use_graph = false;
    G->graph = nullptr;
    G->graph_steps = -1;
    int dev = 0, sms = 152, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_tm2d_group, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGroupStage);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tm2d_group, kGroupThreads, kGroupStage);
    G->grid_blocks = sms * std::max(1, occ);
    if (e == cudaSuccess) e = cudaMemsetAsync(G->ws, 0, L.total, G->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(G->stream);
    if (e != cudaSuccess) {
        delete G;
        return cuda_st(e);
    }
    *out = G;
    return AXP_OK;
}

axp_status axp_group_destroy(axp_group *G)
{
    if (!G) return AXP_E_INVAL;
    for (auto &M : G->members)
        if (M.active) return AXP_E_STATE;  // members must be removed first
    cudaStreamSynchronize(G->stream);
    drop_graph(G);
    delete G;
    return AXP_OK;
}

axp_status axp_group_add(axp_group *G, axp_grid *g, int64_t steps, int32_t *member)
{
    if (!G || !g || !member || steps < 0) return AXP_E_INVAL;
    if (g->group) return AXP_E_STATE;
    if (g->desc.precision != AXP_FP32_SPLIT || g->desc.diag_every != 0 || !tm2d_eligible(g)) return AXP_E_INVAL;
    if (g->src_on) return AXP_E_INVAL;  // member parameters are fixed per parity; a source varies per step
    int m = -1;
    for (int i = 0; i < G->max_grids; i++)
        if (!G->members[i].active) {
            m = i;
            break;
        }
    if (m < 0) return AXP_E_NOMEM;
    int64_t tiles = tiles_of(g, G->chunk);
    for (auto &M : G->members)
        if (M.active) tiles += M.nblk;
    if (tiles > G->max_tiles) return AXP_E_NOMEM;
    // the grid's own pending work, then its fused-path (staggered) state
    cudaError_t e = cudaStreamSynchronize(g->stream);
    if (e == cudaSuccess) e = enter_staggered<float>(g);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_st(e);
    fused::Params<float> P[2];
    P[0] = tm2d_params<float>(g, G->chunk);
    rotate_roles(g);
    P[1] = tm2d_params<float>(g, G->chunk);
    rotate_roles(g);  // period two: back to the present roles
    const int64_t zero = 0;
    const int32_t nblk = tiles_of(g, G->chunk), zero32 = 0;
    e = cudaMemcpyAsync((void *)(G->D.params + 2 * (size_t)m), P, sizeof(P), cudaMemcpyHostToDevice, G->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(G->D.done + m, &zero, sizeof(zero), cudaMemcpyHostToDevice, G->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(G->D.steps + m, &steps, sizeof(steps), cudaMemcpyHostToDevice, G->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(G->D.cnt + m, &zero32, sizeof(zero32), cudaMemcpyHostToDevice, G->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(G->D.nblk + m, &nblk, sizeof(nblk), cudaMemcpyHostToDevice, G->stream);
    // the host sources above must outlive the copies
    if (e == cudaSuccess) e = cudaStreamSynchronize(G->stream);
    if (e != cudaSuccess) return cuda_st(e);
    G->members[m] = axp_group::Member{g, steps, nblk, 1};
    g->group = G;
    g->J_valid = false;
    g->half_prev = false;
    G->dirty = true;
    *member = m;
    return AXP_OK;
}

axp_status axp_group_progress(axp_group *G, int64_t *done, int32_t n)
{
    if (!G || !done || n < 1 || n > G->max_grids) return AXP_E_INVAL;
    cudaError_t e = cudaMemcpyAsync(done, G->D.done, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, G->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(G->stream);
    if (e != cudaSuccess) return cuda_st(e);
    for (int i = 0; i < n; i++)
        if (!G->members[i].active) done[i] = -1;
    return AXP_OK;
}

axp_status axp_group_remove(axp_group *G, int32_t member)
{
    if (!G || member < 0 || member >= G->max_grids || !G->members[member].active) return AXP_E_INVAL;
    int64_t done = 0;
    cudaError_t e = cudaMemcpyAsync(&done, G->D.done + member, sizeof(done), cudaMemcpyDeviceToHost, G->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(G->stream);
    if (e != cudaSuccess) return cuda_st(e);
    axp_grid *g = G->members[member].g;
    if (done & 1) rotate_roles(g);
    g->step += done;
    g->launches += done;
    g->J_valid = false;
    // each group step wrote the other field set from the present one, as a
    // single-grid step does: after one, that set holds E^{n-1/2}
    g->half_prev = done >= 1;
    g->half_prev_cfg = g->cfg_version;
    g->group = nullptr;
    G->members[member] = axp_group::Member{nullptr, 0, 0, 0};
    G->dirty = true;
    return AXP_OK;
}

axp_status axp_group_set_chunk(axp_group *G, int32_t rows)
{
    if (!G || rows < 8 || rows > (1 << 20)) return AXP_E_INVAL;
    for (auto &M : G->members)
        if (M.active) return AXP_E_STATE;  // tiles of present members are fixed
    G->chunk = rows;
    drop_graph(G);
    G->dirty = true;
    return AXP_OK;
}

axp_status axp_group_use_graphs(axp_group *G, int32_t enable)
{
    if (!G) return AXP_E_INVAL;
    if (!enable) drop_graph(G);
    G->use_graph = enable != 0;
    return AXP_OK;
}

axp_status axp_group_launch_count(const axp_group *G, int64_t *count)
{
    if (!G || !count) return AXP_E_INVAL;
    *count = G->launches;
    return AXP_OK;
}

axp_status axp_group_run(axp_group *G, int64_t nsteps)
{
    axp::TraceRange trace_("axp_group_run");
    if (!G || nsteps < 0) return AXP_E_INVAL;
    if (nsteps == 0) return AXP_OK;
    if (G->dirty) {
        drop_graph(G);
        const axp_status st = rebuild(G);
        if (st != AXP_OK) return st;
    }
    if (G->D.nitems == 0) return AXP_OK;
    if (!G->use_graph || G->stream == nullptr) return cuda_st(enqueue(G, nsteps));
    if (!G->graph || G->graph_steps != nsteps) {
        drop_graph(G);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(G->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_st(e);
        const int64_t l0 = G->launches;
        e = enqueue(G, nsteps);
        const cudaError_t e2 = cudaStreamEndCapture(G->stream, &graph);
        G->launches = l0;
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_st(e != cudaSuccess ? e : e2);
        }
        e = cudaGraphInstantiate(&G->graph, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            G->graph = nullptr;
            return cuda_st(e);
        }
        G->graph_steps = nsteps;
    }
    G->launches += nsteps;
    return cuda_st(cudaGraphLaunch(G->graph, G->stream));
}

}  // extern "C"
