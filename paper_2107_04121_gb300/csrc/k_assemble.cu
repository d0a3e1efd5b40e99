// Assembly of element vectors into a global DOF vector (the step after
// Algorithm 1 of Cimrman, arXiv 2107.04121, which Sec. 6 leaves untimed):
//   g[ncomp * conn[e][a] + i] += r[e][i * N + a].
//
// Assembly is done as a gather, not a scatter: the node -> (e, a) incidence
// lists (CSR, ascending element order) are built once per mesh, then one
// thread per global DOF sums its contributions in that fixed order.  No
// floating-point atomics: the result is bit-reproducible and, in FP64, equal to
// a sequential ascending-(e, a) sum.  FP32 sums may be Neumaier-compensated.
#include <mutex>

#include <cub/device/device_scan.cuh>

#include "fe_device.cuh"

namespace {

__global__ void k_count(const int32_t *__restrict__ conn, long long total, long long n_nodes, int *cnt, int *flag)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long node = conn[i];
        if (node < 0 || node >= n_nodes)
            atomicExch(flag, 1);
        else
            atomicAdd(cnt + node, 1);
    }
}

__global__ void k_fill(const int32_t *__restrict__ conn, long long total, long long n_nodes,
                       const int *__restrict__ offsets, int *cursor, int *entries)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long node = conn[i];
        if (node < 0 || node >= n_nodes) continue;
        const int pos = offsets[node] + atomicAdd(cursor + node, 1);
        entries[pos] = (int)i;
    }
}

// Sort each incidence list ascending (lists are short: <= 8 for hex vertices).
__global__ void k_sort(const int *__restrict__ offsets, long long n_nodes, int *entries)
{
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < n_nodes;
         n += (long long)gridDim.x * blockDim.x) {
        const int b = offsets[n], e = offsets[n + 1];
        for (int i = b + 1; i < e; ++i) {
            const int v = entries[i];
            int j = i - 1;
            while (j >= b && entries[j] > v) {
                entries[j + 1] = entries[j];
                --j;
            }
            entries[j + 1] = v;
        }
    }
}

unsigned grid_for(long long n, int threads)
{
    long long b = (n + threads - 1) / threads;
    if (b > 1048576) b = 1048576;
    if (b < 1) b = 1;
    return (unsigned)b;
}

// Assembly by gathering: one thread per node sums, for each of its 1 or 3
// components, the element-vector entries of the node's incidences in ascending
// (e, a) order (the CSR order): deterministic, no atomics; Neumaier-compensated
// in float32 when asked.
template <typename T, bool COMPENSATED, int NC>
__global__ void k_gather_nodes(const int *__restrict__ offsets, const int *__restrict__ entries, long long n_nodes,
                               int N, const T *__restrict__ r, T *__restrict__ out, bool accumulate)
{
    for (long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x; node < n_nodes;
         node += (long long)gridDim.x * blockDim.x) {
        const int b = offsets[node], e = offsets[node + 1];
        T s[NC], c[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            s[k] = accumulate ? out[node * NC + k] : (T)0;
            c[k] = 0;
        }
        for (int p = b; p < e; ++p) {
            const int ent = entries[p];
            const int el = ent / N, a = ent - el * N;
            const T *re = r + (long long)el * NC * N + a;
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                const T x = re[k * N];
                if (COMPENSATED) {
                    const T t = s[k] + x;
                    if (fabs(s[k]) >= fabs(x))
                        c[k] += (s[k] - t) + x;
                    else
                        c[k] += (x - t) + s[k];
                    s[k] = t;
                } else {
                    s[k] += x;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < NC; ++k) out[node * NC + k] = COMPENSATED ? s[k] + c[k] : s[k];
    }
}

template <typename T, bool COMPENSATED>
cudaError_t launch_gather(const fe_assembly_h *a, int ncomp, const void *r, void *out, bool acc, cudaStream_t s)
{
    const long long n_nodes = a->mesh.n_nodes;
    const int N = a->mesh.nodes_per_elem;
    const unsigned grid = grid_for(n_nodes, 256);
    if (ncomp == 3)
        k_gather_nodes<T, COMPENSATED, 3><<<grid, 256, 0, s>>>(a->d_offsets, a->d_entries, n_nodes, N, (const T *)r,
                                                               (T *)out, acc);
    else if (ncomp == 1)
        k_gather_nodes<T, COMPENSATED, 1><<<grid, 256, 0, s>>>(a->d_offsets, a->d_entries, n_nodes, N, (const T *)r,
                                                               (T *)out, acc);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}


}  // namespace

// Builds a->d_offsets / a->d_entries; *d_flag is set to 1 on an out-of-range
// node index.  Temporary buffers are stream-ordered allocations.
cudaError_t fe_launch_assembly_build(fe_assembly_h *a, int *d_flag, cudaStream_t s)
{
    const long long n_nodes = a->mesh.n_nodes, total = a->mesh.n_elems * a->mesh.nodes_per_elem;
    int *cnt = nullptr;
    void *tmp = nullptr;
    size_t tmp_bytes = 0;
    cudaError_t err = cudaMallocAsync((void **)&cnt, sizeof(int) * (n_nodes + 1), s);
    if (err != cudaSuccess) return err;
    err = cudaMemsetAsync(cnt, 0, sizeof(int) * (n_nodes + 1), s);
    if (err == cudaSuccess && total > 0) {
        k_count<<<grid_for(total, 256), 256, 0, s>>>(a->mesh.conn, total, n_nodes, cnt, d_flag);
        err = cudaGetLastError();
    }
    if (err == cudaSuccess)
        err = cub::DeviceScan::ExclusiveSum(nullptr, tmp_bytes, cnt, a->d_offsets, (int)(n_nodes + 1), s);
    if (err == cudaSuccess) err = cudaMallocAsync(&tmp, tmp_bytes > 0 ? tmp_bytes : 16, s);
    if (err == cudaSuccess)
        err = cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, cnt, a->d_offsets, (int)(n_nodes + 1), s);
    if (err == cudaSuccess) err = cudaMemsetAsync(cnt, 0, sizeof(int) * (n_nodes + 1), s);
    if (err == cudaSuccess && total > 0) {
        k_fill<<<grid_for(total, 256), 256, 0, s>>>(a->mesh.conn, total, n_nodes, a->d_offsets, cnt, a->d_entries);
        err = cudaGetLastError();
    }
    if (err == cudaSuccess && n_nodes > 0) {
        k_sort<<<grid_for(n_nodes, 256), 256, 0, s>>>(a->d_offsets, n_nodes, a->d_entries);
        err = cudaGetLastError();
    }
    if (tmp) cudaFreeAsync(tmp, s);
    cudaFreeAsync(cnt, s);
    return err;
}

cudaError_t fe_launch_assemble(const fe_assembly_h *a, int ncomp, bool f64, const void *r, void *out,
                               unsigned flags, cudaStream_t s)
{
    const long long total = a->mesh.n_nodes * ncomp;
    if (total == 0) return cudaSuccess;
    const bool acc = flags & FE_ASSEMBLE_ACCUMULATE;
    if (f64) return launch_gather<double, false>(a, ncomp, r, out, acc, s);
    if (flags & FE_ASSEMBLE_COMPENSATED) return launch_gather<float, true>(a, ncomp, r, out, acc, s);
    return launch_gather<float, false>(a, ncomp, r, out, acc, s);
}

// ---------------------------------------------------------------------------
// One-shot assembly without any device allocation (fe_assemble_vector_noalloc).
// The incidence lists and the counters live in one file-scope device array of
// fixed size, shared by every call on a device and kept until process exit.

namespace {

constexpr long long kNoallocMaxNodes = 1ll << 19;        // 524,288 nodes
constexpr long long kNoallocMaxIncidences = 1ll << 21;   // 2,097,152 (element, local node) pairs
constexpr size_t kNoallocScanBytes = (size_t)1 << 20;    // scan workspace
// each sub-buffer starts on a 256-byte boundary (the scan workspace needs it)
constexpr size_t kNoallocOffsetsBytes = (sizeof(int) * (kNoallocMaxNodes + 1) + 255) / 256 * 256;
constexpr size_t kNoallocScratchBytes =
    2 * kNoallocOffsetsBytes + sizeof(int) * kNoallocMaxIncidences + kNoallocScanBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mutex;
void *g_noalloc_ptr[kNoallocMaxDevices] = {nullptr};

// The host-side symbol is only a stand-in: resolve the device address of the
// array once per device, with that device current.
cudaError_t noalloc_scratch(int device, unsigned char **out)
{
    if (device < 0 || device >= kNoallocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[device]) {
        // the address is per device: resolve it only with `device` current
        int current = -1;
        cudaError_t e = cudaGetDevice(&current);
        if (e != cudaSuccess) return e;
        if (current != device) return cudaErrorInvalidDevice;
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[device] = p;
    }
    *out = (unsigned char *)g_noalloc_ptr[device];
    return cudaSuccess;
}

// Count incidences per node; an out-of-range node index is recorded in the
// context status word (FE_ERR_SHAPE, element index) and skipped.
__global__ void k_count_report(const int32_t *__restrict__ conn, long long total, int N, long long n_nodes, int *cnt,
                               unsigned long long *status)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long node = conn[i];
        if (node < 0 || node >= n_nodes)
            fe_report(status, FE_ERR_SHAPE, i / N);
        else
            atomicAdd(cnt + node, 1);
    }
}

}  // namespace

cudaError_t fe_noalloc_limits(long long n_nodes, long long n_incidences)
{
    return (n_nodes <= kNoallocMaxNodes && n_incidences <= kNoallocMaxIncidences) ? cudaSuccess
                                                                                  : cudaErrorInvalidValue;
}

cudaError_t fe_launch_assemble_noalloc(int device, const fe_mesh *mesh, int ncomp, bool f64, const void *r,
                                       void *out, unsigned flags, unsigned long long *status, cudaStream_t s)
{
    unsigned char *base = nullptr;
    cudaError_t err = noalloc_scratch(device, &base);
    if (err != cudaSuccess) return err;
    const long long n_nodes = mesh->n_nodes, total = mesh->n_elems * mesh->nodes_per_elem;
    int *offsets = (int *)base;
    int *cursor = (int *)(base + kNoallocOffsetsBytes);
    int *entries = (int *)(base + 2 * kNoallocOffsetsBytes);
    void *scan_tmp = base + 2 * kNoallocOffsetsBytes + sizeof(int) * kNoallocMaxIncidences;
    size_t scan_bytes = 0;
    err = cub::DeviceScan::ExclusiveSum(nullptr, scan_bytes, cursor, offsets, (int)(n_nodes + 1), s);
    if (err != cudaSuccess) return err;
    if (scan_bytes > kNoallocScanBytes) return cudaErrorInvalidValue;
    // the array keeps the previous call's contents: counters start from zero
    err = cudaMemsetAsync(cursor, 0, sizeof(int) * (n_nodes + 1), s);
    if (err == cudaSuccess && total > 0) {
        k_count_report<<<grid_for(total, 256), 256, 0, s>>>(mesh->conn, total, mesh->nodes_per_elem, n_nodes, cursor,
                                                            status);
        err = cudaGetLastError();
    }
    if (err == cudaSuccess)
        err = cub::DeviceScan::ExclusiveSum(scan_tmp, scan_bytes, cursor, offsets, (int)(n_nodes + 1), s);
    if (err == cudaSuccess) err = cudaMemsetAsync(cursor, 0, sizeof(int) * (n_nodes + 1), s);
    if (err == cudaSuccess && total > 0) {
        k_fill<<<grid_for(total, 256), 256, 0, s>>>(mesh->conn, total, n_nodes, offsets, cursor, entries);
        err = cudaGetLastError();
    }
    if (err == cudaSuccess && n_nodes > 0) {
        k_sort<<<grid_for(n_nodes, 256), 256, 0, s>>>(offsets, n_nodes, entries);
        err = cudaGetLastError();
    }
    if (err != cudaSuccess) return err;
    fe_assembly_h view{};
    view.device = device;
    view.mesh = *mesh;
    view.d_offsets = offsets;
    view.d_entries = entries;
    return fe_launch_assemble(&view, ncomp, f64, r, out, flags, s);
}
