// Batched matrix mode: element matrices of several (form, element group)
// items, e.g. a mixed mesh of P1-P3 tetrahedra and Q1-Q3 hexahedra with the
// Laplace, mass and elasticity forms of Tab. ewfd (Cimrman, arXiv 2107.04121),
// in ONE persistent launch.
//
// Every item is cut into chunks of EPB consecutive elements; the chunks of all
// items form one work list (item i owns chunks [chunk0_i, chunk0_i + ceil(E_i /
// EPB_i))).  Resident CTAs (a few per SM, 256 threads each) stride over the
// list; each chunk runs the per-element-group body of the SIMT matrix kernel
// (matrix_body.cuh) instantiated for its item's variant: (N, Q) pair, form,
// node tile T, elements per chunk EPB and output staging (bulk row blocks or
// direct stores).  A CTA reloads the reference gradients only when its item
// changes.
//
// Variants per (form, element) are candidates of an autotuner: at plan
// creation each candidate is timed on the item's own elements and the fastest
// is kept.  Registers and shared memory are allocated per kernel, so one kernel
// holding every variant would run all of them at the occupancy of the heaviest
// (Q2 elasticity with 3x3 tiles: 128 registers).  The variants are therefore
// split in three classes, each with its own persistent kernel: "light" (at most
// 80 registers and 75 KB of shared memory: 3 CTAs per SM), "heavy" (2 CTAs per
// SM) and the 4x4-tile Q3 elasticity variant (1 CTA per SM); the three run
// concurrently on three streams (measured faster than one after another).  A
// plan can be captured in a CUDA graph together with the geometry of every
// group (FP64 J, det J, J^-1), so that one graph launch evaluates the whole
// batch.  FP32 element matrices from FP64 geometry.
//
// A second schedule launches, per item, the standalone kernel of
// fe_eval_matrix (each compiled for its item alone, so each runs at its own
// occupancy), the items spread over the caller's stream and the two side
// streams by longest-processing-time-first assignment.  In this schedule an
// item of Lame elasticity or of the scalar Laplacian on 27-node hexahedra may
// take a second contraction path, the TF32x3 Gram on the tensor cores
// (k_matrix_tc), when autotuning finds it faster.  Autotuning times both schedules and keeps the faster; either one
// can be captured in the graph.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "matrix_body.cuh"

namespace {

constexpr int BT = 256;  // threads of the batched kernel

// id, class (0 light / 1 heavy), N, Q, form, material kind (0 scalar / 1 Lame),
// tile T, elements per chunk, staging
#define FE_BATCH_VARIANTS(X)                                      \
    X(0, 0, 4, 5, FK_LAPLACE, 0, 2, 42, STAGE_BULK)               \
    X(1, 0, 4, 5, FK_LAPLACE, 0, 2, 21, STAGE_BULK)               \
    X(2, 0, 4, 5, FK_MASS, 0, 2, 42, STAGE_BULK)                  \
    X(3, 0, 4, 5, FK_MASS, 0, 2, 21, STAGE_BULK)                  \
    X(4, 0, 4, 5, FK_ELASTICITY, 1, 2, 42, STAGE_BULK)            \
    X(5, 0, 4, 5, FK_ELASTICITY, 1, 2, 21, STAGE_BULK)            \
    X(6, 0, 10, 15, FK_LAPLACE, 0, 2, 17, STAGE_BULK)             \
    X(7, 0, 10, 15, FK_LAPLACE, 0, 2, 8, STAGE_BULK)              \
    X(8, 0, 10, 15, FK_MASS, 0, 2, 17, STAGE_BULK)                \
    X(9, 0, 10, 15, FK_MASS, 0, 2, 8, STAGE_BULK)                 \
    X(10, 0, 10, 15, FK_ELASTICITY, 1, 2, 17, STAGE_BULK)         \
    X(11, 0, 10, 15, FK_ELASTICITY, 1, 2, 8, STAGE_BULK)          \
    X(12, 0, 20, 35, FK_LAPLACE, 0, 2, 4, STAGE_BULK)             \
    X(13, 0, 20, 35, FK_LAPLACE, 0, 2, 2, STAGE_BULK)             \
    X(14, 0, 20, 35, FK_MASS, 0, 2, 4, STAGE_BULK)                \
    X(15, 0, 20, 35, FK_MASS, 0, 2, 2, STAGE_BULK)                \
    X(16, 0, 20, 35, FK_ELASTICITY, 1, 2, 4, STAGE_BULK)          \
    X(17, 0, 20, 35, FK_ELASTICITY, 1, 2, 2, STAGE_BULK)          \
    X(18, 0, 8, 8, FK_LAPLACE, 0, 2, 25, STAGE_BULK)              \
    X(19, 0, 8, 8, FK_LAPLACE, 0, 2, 12, STAGE_BULK)              \
    X(20, 0, 8, 8, FK_MASS, 0, 2, 25, STAGE_BULK)                 \
    X(21, 0, 8, 8, FK_MASS, 0, 2, 12, STAGE_BULK)                 \
    X(22, 0, 8, 8, FK_ELASTICITY, 1, 2, 25, STAGE_BULK)           \
    X(23, 0, 8, 8, FK_ELASTICITY, 1, 2, 12, STAGE_BULK)           \
    X(24, 0, 27, 27, FK_LAPLACE, 0, 3, 5, STAGE_BULK)             \
    X(25, 0, 27, 27, FK_LAPLACE, 0, 3, 2, STAGE_BULK)             \
    X(26, 0, 27, 27, FK_MASS, 0, 3, 2, STAGE_BULK)                \
    X(27, 0, 27, 27, FK_MASS, 0, 3, 1, STAGE_BULK)                \
    X(28, 1, 27, 27, FK_ELASTICITY, 1, 3, 5, STAGE_BULK)          \
    X(29, 1, 27, 27, FK_ELASTICITY, 1, 3, 2, STAGE_BULK)          \
    X(30, 1, 64, 64, FK_LAPLACE, 0, 4, 1, STAGE_BULK)             \
    X(31, 1, 64, 64, FK_LAPLACE, 0, 2, 1, STAGE_DIRECT)           \
    X(32, 1, 64, 64, FK_MASS, 0, 4, 1, STAGE_BULK)                \
    X(33, 0, 64, 64, FK_MASS, 0, 2, 1, STAGE_DIRECT)              \
    X(34, 1, 64, 64, FK_ELASTICITY, 1, 2, 1, STAGE_DIRECT)       \
    X(35, 2, 64, 64, FK_ELASTICITY, 1, 4, 1, STAGE_BULK)

struct Variant {
    int cls, N, Q, kind, matk, tile, epb, stage;
    size_t smem;
};

#define FE_BATCH_INFO(ID, CLS, N, Q, KIND, MATK, T, EPB, STAGE) \
    {CLS, N, Q, KIND, MATK, T, EPB, STAGE, MatrixSmem<float, N, Q, KIND, T, EPB, STAGE>::BYTES},
const Variant kVariants[] = {FE_BATCH_VARIANTS(FE_BATCH_INFO)};
#undef FE_BATCH_INFO
constexpr int kNumVariants = (int)(sizeof(kVariants) / sizeof(kVariants[0]));

// shared memory per CTA of each class: 3 (light), 2 (heavy) or 1 (4x4-tile
// elasticity of Q3: 144 accumulators per thread) CTAs per SM
constexpr int kClasses = 3;
constexpr size_t kMaxSmem[kClasses] = {75 * 1024, 113 * 1024, 226 * 1024};  // + the kernel's static bytes <= 227 KB

#define FE_BATCH_CHECK(ID, CLS, N, Q, KIND, MATK, T, EPB, STAGE)                                                 \
    static_assert(STAGE == STAGE_DIRECT || EPB * (N / T) * (N / T + 1) / 2 <= BT, "one tile per thread");      \
    static_assert(MatrixSmem<float, N, Q, KIND, T, EPB, STAGE>::BYTES <= kMaxSmem[CLS], "class cap");
FE_BATCH_VARIANTS(FE_BATCH_CHECK)
#undef FE_BATCH_CHECK

struct BatchItemDev {
    const float *jinv, *wdetj, *dphi, *phi;
    const double *mat;
    float *K;
    long long E;
    long long chunk0;  // first chunk of this item in the work list
    int variant, ncomp, mat_t, pad;
};

template <int CLS>
__global__ void __launch_bounds__(BT, CLS == 0 ? 3 : (CLS == 1 ? 2 : 1)) k_batch(const BatchItemDev *__restrict__ items, int n_items,
                                                           long long n_chunks)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    int loaded = -1;  // item whose reference gradients are in shared memory
    for (long long c = blockIdx.x; c < n_chunks; c += gridDim.x) {
        if (threadIdx.x == 0) {
            int lo = 0, hi = n_items - 1;  // last item with chunk0 <= c
            while (lo < hi) {
                const int mid = (lo + hi + 1) / 2;
                if (items[mid].chunk0 <= c) lo = mid;
                else hi = mid - 1;
            }
            s_item = lo;
        }
        __syncthreads();
        const int i = s_item;
        const BatchItemDev it = items[i];
        const long long local = c - it.chunk0;
        if (i != loaded) {
            // another variant's plan may alias this one: earlier bulk copies must
            // have finished reading shared memory before it is rewritten
            if (threadIdx.x == 0) bulk_wait_read<0>();
            __syncthreads();
        }
        switch (it.variant) {
#define FE_BATCH_CASE(ID, VCLS, N, Q, KIND, MATK, T, EPB, STAGE)                                                 \
    case ID:                                                                                                    \
        if constexpr (VCLS == CLS) {                                                                            \
            if (i != loaded) matrix_load_ref<float, N, Q, KIND, T, EPB, BT, STAGE>(it.dphi, smem_raw);          \
            const long long e0 = local * EPB;                                                                   \
            const int ne = (int)(it.E - e0 < EPB ? it.E - e0 : EPB);                                             \
            matrix_group<float, N, Q, KIND, MATK, T, EPB, BT, STAGE>(it.jinv, it.wdetj, it.phi, it.dphi, e0, ne,         \
                                                                     it.ncomp, it.mat, it.mat_t, it.K, smem_raw); \
        }                                                                                                       \
        break;
            FE_BATCH_VARIANTS(FE_BATCH_CASE)
#undef FE_BATCH_CASE
        default: break;
        }
        loaded = i;
        __syncthreads();  // every thread has read s_item before it is rewritten
    }
    if (threadIdx.x == 0) bulk_wait_read<0>();  // shared memory must outlive the copies' reads
}

// Launch shape of class CLS for a shared-memory plan of `smem` bytes.
template <int CLS>
cudaError_t batch_grid(size_t smem, long long *grid)
{
    static FeLaunchCache cache;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    long long set = 0;
    e = fe_cached_grid(
        cache,
        [&](int, long long *v) {
            *v = 1;
            cudaError_t e2 = cudaFuncSetAttribute(k_batch<CLS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)kMaxSmem[CLS]);
            if (e2 != cudaSuccess) return e2;
            // the whole carveout as shared memory, so that the occupancy below counts
            // every CTA the shared memory of an SM holds
            return cudaFuncSetAttribute(k_batch<CLS>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        },
        &set);
    if (e != cudaSuccess) return e;
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<CLS>, BT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    *grid = (long long)per_sm * sms;
    return cudaSuccess;
}

cudaError_t launch_class(int cls, const BatchItemDev *items, int n, long long chunks, size_t smem, long long grid,
                         cudaStream_t s)
{
    if (n == 0 || chunks == 0) return cudaSuccess;
    if (grid > chunks) grid = chunks;
    if (cls == 0) k_batch<0><<<(unsigned)grid, BT, smem, s>>>(items, n, chunks);
    else if (cls == 1) k_batch<1><<<(unsigned)grid, BT, smem, s>>>(items, n, chunks);
    else k_batch<2><<<(unsigned)grid, BT, smem, s>>>(items, n, chunks);
    return cudaGetLastError();
}

}  // namespace

struct fe_batch_h {
    int device;
    int n_items;
    unsigned flags;
    unsigned long long *d_status;
    std::vector<BatchItemDev> items;     // in the caller's order; chunk0 relative to the item's class
    std::vector<int> pos;                // device position of each item (grouped by class)
    std::vector<fe_geometry_h *> geoms;  // distinct geometries recomputed by the batch
    BatchItemDev *d_items = nullptr;
    int n_cls[kClasses] = {0, 0, 0};
    int first[kClasses] = {0, 0, 0};  // device position of each class's first item
    long long chunks[kClasses] = {0, 0, 0};
    size_t smem[kClasses] = {0, 0, 0};
    long long grid[kClasses] = {0, 0, 0};
    cudaStream_t side[kClasses - 1] = {nullptr, nullptr};  // classes 1, 2 run here, concurrently
    cudaEvent_t fork = nullptr, join[kClasses - 1] = {nullptr, nullptr};
    cudaStream_t capture_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // per-item schedule: fe_eval_matrix's kernel for every item on its lane
    // (0: the caller's stream, 1 and 2: the side streams)
    int launches = 0;
    int sm_count = 0;
    std::vector<const fe_form_h *> forms;
    std::vector<const fe_geometry_h *> igeom;
    std::vector<fe_material_args> mats;
    std::vector<int> lane;
    // contraction path of each item in the per-item schedule: 0 the Gram blocks on
    // the CUDA cores (k_matrix_sym), 1 the TF32x3 Gram on the tensor cores
    // (k_matrix_tc; Lame elasticity and the scalar Laplacian of 27-node
    // hexahedra with 27 points)
    std::vector<int> path;
    // shared Gram blocks (per-item schedule): a Lame elasticity item and a scalar
    // Laplacian item on the same geometry computed by one CUDA-core launch, the
    // Laplacian as c sum_j A_jj of the elasticity's Gram blocks; partner index or -1
    std::vector<int> pair;
    // per-item schedule with FE_BATCH_GEOMETRY: the lane that recomputes each
    // geometry (that of its largest item) and the event the other lanes wait on
    std::vector<int> geo_lane;
    std::vector<cudaEvent_t> geo_done;
};

namespace {

// Matrices, persistent schedule: class 0 on the caller's stream, classes 1
// and 2 forked onto the side streams.
cudaError_t enqueue_persistent(fe_batch_h *b, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    int used = 0;
    for (int c = 1; c < kClasses; ++c) used += b->chunks[c] > 0;
    if (used > 0) {
        e = cudaEventRecord(b->fork, s);
        for (int c = 1; c < kClasses && e == cudaSuccess; ++c) {
            if (b->chunks[c] == 0) continue;
            e = cudaStreamWaitEvent(b->side[c - 1], b->fork, 0);
            if (e == cudaSuccess)
                e = launch_class(c, b->d_items + b->first[c], b->n_cls[c], b->chunks[c], b->smem[c], b->grid[c],
                                 b->side[c - 1]);
        }
    }
    if (e == cudaSuccess)
        e = launch_class(0, b->d_items + b->first[0], b->n_cls[0], b->chunks[0], b->smem[0], b->grid[0], s);
    for (int c = 1; c < kClasses && e == cudaSuccess; ++c) {
        if (b->chunks[c] == 0) continue;
        e = cudaEventRecord(b->join[c - 1], b->side[c - 1]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->join[c - 1], 0);
    }
    return e;
}

// Item i's kernel in the per-item schedule: fe_eval_matrix's kernel on its path, or,
// for a shared-Gram pair, one launch from the elasticity item on its path (CUDA
// cores, or the tensor cores for 27- and 64-node hexahedra; the Laplacian item
// launches nothing).
cudaError_t launch_item(fe_batch_h *b, int i, cudaStream_t s)
{
    const int j = b->pair[i];
    if (j >= 0) {
        if (b->forms[i]->kind != FK_ELASTICITY) return cudaSuccess;
        return b->path[i] ? fe_launch_matrix_tc_pair(b->igeom[i], b->mats[i].data, b->items[i].K, b->mats[j].data,
                                                      b->items[j].K, b->sm_count, b->d_status, s)
                          : fe_launch_matrix_pair(b->igeom[i], b->mats[i].data, b->items[i].K, b->mats[j].data,
                                                  b->items[j].K, b->sm_count, s);
    }
    return b->path[i] ? fe_launch_matrix_tc(b->igeom[i], b->forms[i], b->mats[i], FE_TF32X3, b->items[i].K,
                                            b->sm_count, b->d_status, nullptr, false, s)
                      : fe_launch_matrix_simt(b->igeom[i], b->forms[i], b->mats[i], false, b->items[i].K,
                                              b->sm_count, s);
}

// Index of item i's geometry in b->geoms.
int geo_index(const fe_batch_h *b, int i)
{
    for (size_t k = 0; k < b->geoms.size(); ++k)
        if (b->geoms[k] == b->igeom[i]) return (int)k;
    return -1;
}

// Matrices, per-item schedule: each item's fe_eval_matrix kernel on its lane.  With
// `geometry`, each geometry is recomputed first on its own lane, and an item on
// another lane waits for it, so that one group's geometry overlaps the matrices of
// the groups already done.
cudaError_t enqueue_items(fe_batch_h *b, cudaStream_t s, bool geometry = false)
{
    cudaError_t e = cudaEventRecord(b->fork, s);
    for (int c = 0; c < kClasses - 1 && e == cudaSuccess; ++c) e = cudaStreamWaitEvent(b->side[c], b->fork, 0);
    auto lane_stream = [&](int l) { return l == 0 ? s : b->side[l - 1]; };
    if (geometry)
        for (size_t k = 0; k < b->geoms.size() && e == cudaSuccess; ++k) {
            fe_geometry_h *g = b->geoms[k];
            g->pending = 0;
            e = fe_launch_geometry(g, b->d_status, lane_stream(b->geo_lane[k]));
            if (e == cudaSuccess) e = cudaEventRecord(b->geo_done[k], lane_stream(b->geo_lane[k]));
        }
    for (int i = 0; i < b->n_items && e == cudaSuccess; ++i) {
        if (b->items[i].E == 0) continue;
        const int l = b->lane[i];
        cudaStream_t ls = lane_stream(l);
        if (geometry) {
            // the geometry of the item (and, for a shared-Gram pair, of its partner: the same)
            const int k = geo_index(b, i);
            if (k >= 0 && b->geo_lane[k] != l) e = cudaStreamWaitEvent(ls, b->geo_done[k], 0);
            if (e != cudaSuccess) break;
        }
        e = launch_item(b, i, ls);
    }
    for (int c = 0; c < kClasses - 1 && e == cudaSuccess; ++c) {
        e = cudaEventRecord(b->join[c], b->side[c]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->join[c], 0);
    }
    return e;
}

cudaError_t enqueue_matrices(fe_batch_h *b, cudaStream_t s)
{
    return b->launches ? enqueue_items(b, s) : enqueue_persistent(b, s);
}

cudaError_t enqueue(fe_batch_h *b, cudaStream_t s)
{
    if ((b->flags & FE_BATCH_GEOMETRY) && b->launches) return enqueue_items(b, s, true);
    if (b->flags & FE_BATCH_GEOMETRY)
        for (fe_geometry_h *g : b->geoms) {
            g->pending = 0;
            const cudaError_t e = fe_launch_geometry(g, b->d_status, s);
            if (e != cudaSuccess) return e;
        }
    return enqueue_matrices(b, s);
}

// Median of three timed runs (after one warm-up) of the batch's matrix launches
// under its current schedule.
cudaError_t time_schedule(fe_batch_h *b, cudaStream_t s, float *ms)
{
    cudaEvent_t a, z;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&z);
    if (e != cudaSuccess) {
        cudaEventDestroy(a);
        return e;
    }
    float t[3] = {0.f, 0.f, 0.f};
    for (int r = 0; r < 4 && e == cudaSuccess; ++r) {
        e = cudaEventRecord(a, s);
        if (e == cudaSuccess) e = enqueue_matrices(b, s);
        if (e == cudaSuccess) e = cudaEventRecord(z, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(z);
        if (e == cudaSuccess && r > 0) e = cudaEventElapsedTime(&t[r - 1], a, z);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(z);
    std::sort(t, t + 3);
    *ms = t[1];
    return e;
}

// Candidate variants of an item: same element pair, form and material kind.
std::vector<int> candidates(int N, int Q, int kind, int matk)
{
    std::vector<int> v;
    for (int id = 0; id < kNumVariants; ++id) {
        const Variant &x = kVariants[id];
        if (x.N == N && x.Q == Q && x.kind == kind && x.matk == matk) v.push_back(id);
    }
    return v;
}

cudaError_t class_grid(int cls, size_t smem, long long *grid)
{
    return cls == 0 ? batch_grid<0>(smem, grid) : cls == 1 ? batch_grid<1>(smem, grid) : batch_grid<2>(smem, grid);
}

// Median of five timed runs (after one warm-up) of one item alone with variant `id`.
cudaError_t time_variant(BatchItemDev it, int id, BatchItemDev *d_tmp, cudaStream_t s, float *ms)
{
    const Variant &v = kVariants[id];
    it.variant = id;
    it.chunk0 = 0;
    const long long chunks = (it.E + v.epb - 1) / v.epb;
    long long grid = 0;
    cudaError_t e = class_grid(v.cls, v.smem, &grid);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(d_tmp, &it, sizeof(it), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float t[5];
    for (int r = 0; r < 6; ++r) {
        cudaEventRecord(a, s);
        e = launch_class(v.cls, d_tmp, 1, chunks, v.smem, grid, s);
        cudaEventRecord(b, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        if (e != cudaSuccess) break;
        if (r > 0) cudaEventElapsedTime(&t[r - 1], a, b);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return e;
    for (int i = 1; i < 5; ++i)
        for (int j = i; j > 0 && t[j] < t[j - 1]; --j) {
            const float x = t[j];
            t[j] = t[j - 1];
            t[j - 1] = x;
        }
    *ms = t[2];
    return cudaSuccess;
}

// Median of five timed runs (after one warm-up) of item i's kernel in the per-item
// schedule with path `path` (0 CUDA cores, 1 tensor cores) and partner `partner`
// (a shared-Gram pair when >= 0).
cudaError_t time_path(fe_batch_h *b, int i, int path, int partner, cudaStream_t s, float *ms)
{
    const int keep_path = b->path[i], keep_pair = b->pair[i];
    b->path[i] = path;
    b->pair[i] = partner;
    cudaEvent_t a, z;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&z);
    if (e != cudaSuccess) {
        cudaEventDestroy(a);
        return e;
    }
    float t[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (int r = 0; r < 6 && e == cudaSuccess; ++r) {
        e = cudaEventRecord(a, s);
        if (e == cudaSuccess) e = launch_item(b, i, s);
        if (e == cudaSuccess) e = cudaEventRecord(z, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(z);
        if (e == cudaSuccess && r > 0) e = cudaEventElapsedTime(&t[r - 1], a, z);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(z);
    b->path[i] = keep_path;
    b->pair[i] = keep_pair;
    std::sort(t, t + 5);
    *ms = t[2];
    return e;
}

void free_plan(fe_batch_h *b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    for (int c = 0; c < kClasses - 1; ++c) {
        if (b->side[c]) cudaStreamDestroy(b->side[c]);
        if (b->join[c]) cudaEventDestroy(b->join[c]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    for (cudaEvent_t ev : b->geo_done)
        if (ev) cudaEventDestroy(ev);
    if (b->d_items) cudaFree(b->d_items);
    delete b;
}

}  // namespace

extern "C" {

fe_status fe_batch_create(fe_ctx *ctx, const fe_batch_item *items, int n_items, unsigned flags, fe_batch_h **out,
                          fe_stream_t stream)
{
    fe_clear_last_error();
    if (!ctx || !out || n_items < 1 || !items) return FE_ERR_INVALID_ARG;
    if (flags & ~(FE_BATCH_GEOMETRY | FE_BATCH_AUTOTUNE | FE_BATCH_GRAPH | FE_BATCH_PERSISTENT | FE_BATCH_LAUNCHES |
                  FE_BATCH_SHARED_GRAM))
        return FE_ERR_INVALID_ARG;
    const bool force_persistent = flags & FE_BATCH_PERSISTENT, force_launches = flags & FE_BATCH_LAUNCHES;
    if (force_persistent && force_launches) return FE_ERR_INVALID_ARG;
    *out = nullptr;
    cudaSetDevice(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    fe_batch_h *b = new (std::nothrow) fe_batch_h();
    if (!b) return FE_ERR_OOM;
    b->device = ctx->device;
    b->n_items = n_items;
    b->flags = flags;
    b->d_status = ctx->d_status;
    b->sm_count = ctx->sm_count;
    b->launches = force_launches ? 1 : 0;
    // validate and describe the items
    std::vector<std::vector<int>> cand(n_items);
    for (int i = 0; i < n_items; ++i) {
        const fe_batch_item &x = items[i];
        const fe_geometry_h *g = x.geom;
        const fe_form_h *f = x.form;
        fe_status bad = FE_OK;
        int matk = 0;
        if (!g || !f || g->device != ctx->device) bad = FE_ERR_INVALID_ARG;
        else if (g->mesh.n_elems > 0 && !x.K_out) bad = FE_ERR_INVALID_ARG;
        else if (!g->d_jinv32) bad = FE_ERR_INVALID_ARG;  // the batch reads the FP32 copy of the geometry
        else if (f->eval) bad = FE_ERR_INVALID_ARG;
        else if (f->kind == FK_LAPLACE || f->kind == FK_MASS) matk = 0;
        else if (f->kind == FK_ELASTICITY && f->mat == FE_MAT_LAME && !f->mat_transposed) matk = 1;
        else bad = FE_ERR_UNSUPPORTED_SPEC;
        if (bad == FE_OK && f->mat_op >= 0 && !x.material && g->mesh.n_elems > 0) bad = FE_ERR_INVALID_ARG;
        if (bad == FE_OK) {
            cand[i] = candidates(g->N, g->Q, f->kind, matk);
            if (cand[i].empty()) bad = FE_ERR_UNSUPPORTED_SPEC;
        }
        if (bad != FE_OK) {
            free_plan(b);
            return bad;
        }
        BatchItemDev it{};
        it.jinv = g->d_jinv32;
        it.wdetj = g->d_wdetj32;
        it.dphi = g->d_dphi32;
        it.phi = g->d_phi32;
        it.mat = f->mat_op >= 0 ? (const double *)x.material : nullptr;
        it.K = (float *)x.K_out;
        it.E = g->mesh.n_elems;
        it.variant = cand[i][0];
        it.ncomp = f->ncomp;
        it.mat_t = f->mat_transposed;
        b->items.push_back(it);
        b->forms.push_back(f);
        b->igeom.push_back(g);
        fe_material_args ma{};
        ma.kind = f->mat_op >= 0 ? f->mat : FE_MAT_NONE;
        ma.data = f->mat_op >= 0 ? (const double *)x.material : nullptr;
        ma.transposed = f->mat_op >= 0 ? f->mat_transposed : 0;
        b->mats.push_back(ma);
        b->path.push_back(0);
        b->pair.push_back(-1);
        fe_geometry_h *gm = const_cast<fe_geometry_h *>(g);
        bool seen = false;
        for (fe_geometry_h *h : b->geoms) seen = seen || h == gm;
        if (!seen) b->geoms.push_back(gm);
    }
    cudaError_t e = cudaMalloc(&b->d_items, sizeof(BatchItemDev) * (size_t)n_items);
    for (int c = 0; c < kClasses - 1 && e == cudaSuccess; ++c) {
        e = cudaStreamCreateWithFlags(&b->side[c], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[c], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    // geometry first (stale deferred handles)
    for (fe_geometry_h *g : b->geoms)
        if (e == cudaSuccess) e = fe_settle_geometry(g, ctx->d_status, s);
    // autotune: time every candidate on each item alone; items of the same
    // (element, form, components) share the result
    if (e == cudaSuccess && (flags & FE_BATCH_AUTOTUNE) && !force_launches) {
        struct Key {
            int N, Q, kind, ncomp, variant;
        };
        std::vector<Key> done;
        for (int i = 0; i < n_items && e == cudaSuccess; ++i) {
            BatchItemDev &it = b->items[i];
            if (it.E == 0 || cand[i].size() < 2) continue;
            const fe_geometry_h *g = items[i].geom;
            int found = -1;
            for (const Key &k : done)
                if (k.N == g->N && k.Q == g->Q && k.kind == items[i].form->kind && k.ncomp == it.ncomp)
                    found = k.variant;
            if (found >= 0) {
                it.variant = found;
                continue;
            }
            float best = 0.f;
            int best_id = cand[i][0];
            for (size_t c = 0; c < cand[i].size() && e == cudaSuccess; ++c) {
                float ms = 0.f;
                e = time_variant(it, cand[i][c], b->d_items, s, &ms);
                if (e == cudaSuccess && (c == 0 || ms < best)) {
                    best = ms;
                    best_id = cand[i][c];
                }
            }
            it.variant = best_id;
            done.push_back({g->N, g->Q, items[i].form->kind, it.ncomp, best_id});
        }
    }
    // contraction path per item (per-item schedule): the tensor-core TF32x3 Gram
    // where it applies and runs faster than the CUDA-core kernel
    if (e == cudaSuccess && (flags & FE_BATCH_AUTOTUNE) && !force_persistent) {
        for (int i = 0; i < n_items && e == cudaSuccess; ++i) {
            const fe_geometry_h *g = b->igeom[i];
            const fe_form_h *f = b->forms[i];
            if (b->items[i].E == 0 || !fe_matrix_tc_supported(g, f, FE_TF32X3)) continue;
            float t0 = 0.f, t1 = 0.f;
            e = time_path(b, i, 0, -1, s, &t0);
            if (e == cudaSuccess) e = time_path(b, i, 1, -1, s, &t1);
            if (e == cudaSuccess && t1 < t0) b->path[i] = 1;
        }
    }
    // shared Gram blocks: a Lame elasticity item and a scalar Laplacian item on the
    // same geometry in one launch, where that beats the two items' chosen kernels
    // (timed), or always with FE_BATCH_SHARED_GRAM
    const bool share_all = flags & FE_BATCH_SHARED_GRAM;
    if (e == cudaSuccess && !force_persistent && ((flags & FE_BATCH_AUTOTUNE) || share_all)) {
        for (int i = 0; i < n_items && e == cudaSuccess; ++i) {
            const fe_form_h *f = b->forms[i];
            if (b->items[i].E == 0 || f->kind != FK_ELASTICITY || b->mats[i].kind != FE_MAT_LAME ||
                b->mats[i].transposed || !fe_matrix_pair_supported(b->igeom[i]))
                continue;
            int j = -1;
            for (int k = 0; k < n_items && j < 0; ++k)
                if (b->pair[k] < 0 && b->igeom[k] == b->igeom[i] && b->forms[k]->kind == FK_LAPLACE &&
                    b->forms[k]->ncomp == 1)
                    j = k;
            if (j < 0) continue;
            const bool tc_pair = fe_matrix_tc_pair_supported(b->igeom[i]);
            if (share_all) {  // on the tensor cores where a shared kernel exists
                b->pair[i] = j;
                b->pair[j] = i;
                b->path[i] = tc_pair ? 1 : 0;
                continue;
            }
            float ti = 0.f, tj = 0.f, tp = 0.f, tq = 0.f;
            e = time_path(b, i, b->path[i], -1, s, &ti);
            if (e == cudaSuccess) e = time_path(b, j, b->path[j], -1, s, &tj);
            if (e == cudaSuccess) e = time_path(b, i, 0, j, s, &tp);
            if (e == cudaSuccess && tc_pair) e = time_path(b, i, 1, j, s, &tq);
            const bool use_tc = tc_pair && tq < tp;
            if (e == cudaSuccess && (use_tc ? tq : tp) < ti + tj) {
                b->pair[i] = j;
                b->pair[j] = i;
                b->path[i] = use_tc ? 1 : 0;
            }
        }
    }
    // work lists: one per class, the items grouped by class on the device
    std::vector<BatchItemDev> dev;
    b->pos.assign(n_items, 0);
    for (int cls = 0; cls < kClasses; ++cls) {
        b->first[cls] = (int)dev.size();
        for (int i = 0; i < n_items; ++i) {
            BatchItemDev &it = b->items[i];
            const Variant &v = kVariants[it.variant];
            if (v.cls != cls) continue;
            it.chunk0 = b->chunks[cls];
            b->chunks[cls] += (it.E + v.epb - 1) / v.epb;
            if (it.E > 0 && v.smem > b->smem[cls]) b->smem[cls] = v.smem;
            b->pos[i] = (int)dev.size();
            dev.push_back(it);
            ++b->n_cls[cls];
        }
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_items, dev.data(), sizeof(BatchItemDev) * (size_t)n_items, cudaMemcpyHostToDevice, s);
    for (int cls = 0; cls < kClasses && e == cudaSuccess; ++cls)
        if (b->chunks[cls] > 0) e = class_grid(cls, b->smem[cls] > 0 ? b->smem[cls] : 1024, &b->grid[cls]);
    // lanes of the per-item schedule: largest first, each to the least loaded
    // stream (work ~ bytes of K written + float32 geometry read)
    {
        std::vector<int> order(n_items);
        std::vector<double> cost(n_items);
        for (int i = 0; i < n_items; ++i) {
            const fe_geometry_h *g = b->igeom[i];
            const double n = (double)b->forms[i]->ncomp * g->N;
            cost[i] = (double)b->items[i].E * (4.0 * n * n + 40.0 * g->Q);
            order[i] = i;
        }
        // a shared-Gram pair runs as one launch on the elasticity item's lane
        for (int i = 0; i < n_items; ++i)
            if (b->pair[i] >= 0 && b->forms[i]->kind == FK_LAPLACE) {
                cost[b->pair[i]] += cost[i];
                cost[i] = 0.0;
            }
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
        double load[kClasses] = {0.0, 0.0, 0.0};
        b->lane.assign(n_items, 0);
        for (int i : order) {
            int l = 0;
            for (int c = 1; c < kClasses; ++c)
                if (load[c] < load[l]) l = c;
            b->lane[i] = l;
            load[l] += cost[i];
        }
        // each geometry on the lane of its largest item
        b->geo_lane.assign(b->geoms.size(), -1);
        for (int i : order) {
            const int k = geo_index(b, i);
            if (k >= 0 && b->geo_lane[k] < 0) b->geo_lane[k] = b->lane[i];
        }
        for (int &l : b->geo_lane)
            if (l < 0) l = 0;
        b->geo_done.assign(b->geoms.size(), nullptr);
        for (size_t k = 0; k < b->geoms.size() && e == cudaSuccess; ++k)
            e = cudaEventCreateWithFlags(&b->geo_done[k], cudaEventDisableTiming);
    }
    // schedule: fixed by a flag, else timed when autotuning (matrix launches only)
    if (e == cudaSuccess && !force_persistent && !force_launches && (flags & FE_BATCH_AUTOTUNE)) {
        float t[2] = {0.f, 0.f};
        for (int mode = 0; mode < 2 && e == cudaSuccess; ++mode) {
            b->launches = mode;
            e = time_schedule(b, s, &t[mode]);
        }
        b->launches = t[1] < t[0] ? 1 : 0;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    // CUDA graph of the whole batch, captured on a private stream
    if (e == cudaSuccess && (flags & FE_BATCH_GRAPH)) {
        e = enqueue(b, s);  // one eager run: first-launch attributes are set outside the capture
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t e1 = enqueue(b, b->capture_stream);
            const cudaError_t e2 = cudaStreamEndCapture(b->capture_stream, &b->graph);
            e = e1 != cudaSuccess ? e1 : e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    }
    if (e != cudaSuccess) {
        fe_status st = fe_status_from_cuda(e, "fe_batch_create");
        free_plan(b);
        return st;
    }
    *out = b;
    return FE_OK;
}

fe_status fe_batch_run(fe_ctx *ctx, fe_batch_h *batch, fe_stream_t stream)
{
    fe_clear_last_error();
    if (!ctx || !batch || batch->device != ctx->device) return FE_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (batch->exec) {
        for (fe_geometry_h *g : batch->geoms) g->pending = 0;
        e = cudaGraphLaunch(batch->exec, s);
    } else {
        e = cudaSuccess;
        if (!(batch->flags & FE_BATCH_GEOMETRY))
            for (fe_geometry_h *g : batch->geoms)
                if (e == cudaSuccess) e = fe_settle_geometry(g, batch->d_status, s);
        if (e == cudaSuccess) e = enqueue(batch, s);
    }
    return fe_status_from_cuda(e, "fe_batch_run");
}

fe_status fe_batch_describe(const fe_batch_h *batch, int item, int *tile, int *elems_per_chunk, int *staging)
{
    fe_clear_last_error();
    if (!batch || item < 0 || item >= batch->n_items) return FE_ERR_INVALID_ARG;
    const Variant &v = kVariants[batch->items[item].variant];
    if (tile) *tile = v.tile;
    if (elems_per_chunk) *elems_per_chunk = v.epb;
    if (staging) *staging = v.stage == STAGE_BULK ? 1 : 0;
    return FE_OK;
}

fe_status fe_batch_describe_path(const fe_batch_h *batch, int item, int *path)
{
    fe_clear_last_error();
    if (!batch || !path || item < 0 || item >= batch->n_items) return FE_ERR_INVALID_ARG;
    const int partner = batch->pair[item];
    if (!batch->launches) *path = 0;
    else if (partner < 0) *path = batch->path[item];
    else *path = 2 + batch->path[batch->forms[item]->kind == FK_ELASTICITY ? item : partner];
    return FE_OK;
}

fe_status fe_batch_schedule(const fe_batch_h *batch, int *per_item_launches)
{
    fe_clear_last_error();
    if (!batch || !per_item_launches) return FE_ERR_INVALID_ARG;
    *per_item_launches = batch->launches;
    return FE_OK;
}

fe_status fe_batch_free(fe_batch_h *batch)
{
    fe_clear_last_error();
    if (!batch) return FE_ERR_INVALID_ARG;
    cudaSetDevice(batch->device);
    free_plan(batch);
    return FE_OK;
}

}  // extern "C"
