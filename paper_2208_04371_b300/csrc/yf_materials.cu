// Edge-material classes from the per-cell material index (Sec. II-B, III: dielectrics
// and lossy metals; the interface rule is this library's reading, the paper is silent).
//
// Each interior E edge is shared by four cells; it takes the mean eps_r and sigma of
// those cells and is PEC if any of them is PEC.  Edges on the domain walls are
// tangential to a wall and held at zero (class 0).  The multiset of the four material
// ids identifies an edge's material, so the GPU collects the distinct sorted id
// quadruples in a small hash set, the host turns each into (eps, sigma) and numbers the
// distinct pairs 1..255 in sorted order (deterministic), and a second pass writes the
// uint8 class of every edge.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <utility>
#include <vector>

#include "yf_internal.h"

namespace yf {
namespace {

constexpr int kHashBits = 14;
constexpr int kHashSize = 1 << kHashBits;
constexpr uint32_t kEmpty = 0xFFFFFFFFu;   // also the key of a PEC edge (never inserted)

struct KeyArgs {
    const uint8_t *ids;
    const uint8_t *pec;   // [256]
    int nmat;
    int *overflow;        // bit 0: hash set full, bit 1: id >= nmat
    int nx, ny, nz, px;
    long plane;
};

__device__ __forceinline__ void cswap(uint32_t &a, uint32_t &b)
{
    const uint32_t lo = min(a, b), hi = max(a, b);
    a = lo; b = hi;
}

// The material ids of the cells around node (i, j, k) at offsets (di, dj, dk) in {-1, 0}^3:
// the three E edges of the node use seven of the eight (all but (-1, -1, -1)); a cell outside
// the grid reads as 0 and is never used (its edges are walls).
struct NodeCells {
    uint32_t c000, c100, c010, c001, c110, c101, c011;   // c<-di><-dj><-dk>: 1 = offset -1
};

__device__ __forceinline__ NodeCells node_cells(const KeyArgs &A, int i, int j, int k)
{
    const long sy = A.nx, sz = (long)A.nx * A.ny;
    const long c = (long)k * sz + (long)j * sy + i;
    const bool in = i < A.nx && j < A.ny && k < A.nz;
    const bool im = i >= 1, jm = j >= 1, km = k >= 1;
    const bool xi = i < A.nx && i >= 0, yj = j < A.ny, zk = k < A.nz;
    NodeCells n;
    n.c000 = in ? A.ids[c] : 0;
    n.c100 = (im && yj && zk) ? A.ids[c - 1] : 0;
    n.c010 = (xi && jm && zk) ? A.ids[c - sy] : 0;
    n.c001 = (xi && yj && km) ? A.ids[c - sz] : 0;
    n.c110 = (im && jm && zk) ? A.ids[c - 1 - sy] : 0;
    n.c101 = (im && yj && km) ? A.ids[c - 1 - sz] : 0;
    n.c011 = (xi && jm && km) ? A.ids[c - sy - sz] : 0;
    return n;
}

// the four cell ids of edge `comp` at node (i, j, k); false for wall and non-existent edges
__device__ __forceinline__ bool edge_ids(const KeyArgs &A, const NodeCells &n, int comp, int i, int j, int k,
                                         uint32_t id[4])
{
    if (comp == 0) {            // E_x(i+1/2, j, k): cells at dj, dk in {-1, 0}
        if (i >= A.nx || j < 1 || j >= A.ny || k < 1 || k >= A.nz) return false;
        id[0] = n.c011; id[1] = n.c001; id[2] = n.c010; id[3] = n.c000;
    } else if (comp == 1) {     // E_y(i, j+1/2, k): cells at di, dk in {-1, 0}
        if (i < 1 || i >= A.nx || j >= A.ny || k < 1 || k >= A.nz) return false;
        id[0] = n.c101; id[1] = n.c001; id[2] = n.c100; id[3] = n.c000;
    } else {                    // E_z(i, j, k+1/2): cells at di, dj in {-1, 0}
        if (i < 1 || i >= A.nx || j < 1 || j >= A.ny || k >= A.nz) return false;
        id[0] = n.c110; id[1] = n.c010; id[2] = n.c100; id[3] = n.c000;
    }
    return true;
}

__device__ __forceinline__ bool uniform(const uint32_t id[4]) { return id[0] == id[1] && id[1] == id[2] && id[2] == id[3]; }

// key of an edge from its four cell ids: kEmpty when one of them is PEC (pec is the block's
// shared copy of the per-material flags)
__device__ __forceinline__ uint32_t key_of(const KeyArgs &A, const uint8_t *pec, uint32_t id[4])
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if ((int)id[q] >= A.nmat) { atomicOr(A.overflow, 2); return kEmpty; }
        if (pec[id[q]]) return kEmpty;
    }
    cswap(id[0], id[1]); cswap(id[2], id[3]); cswap(id[0], id[2]); cswap(id[1], id[3]);
    cswap(id[1], id[2]);
    return id[0] | (id[1] << 8) | (id[2] << 16) | (id[3] << 24);
}

__device__ __forceinline__ uint32_t hash_slot(uint32_t key)
{
    return (key * 2654435761u) >> (32 - kHashBits);
}

constexpr int kCache = 64;   // per-block direct-mapped cache of keys (classes) already handled

// Both passes run over nodes (i, j, k): a block's threads stride along the row i, blocks
// stride over rows j (grid y) and planes k (grid z); about a thousand resident blocks, so that
// each keeps its caches over many rows.
__device__ __forceinline__ void load_pec(const KeyArgs &A, uint8_t *pec)
{
    for (int q = threadIdx.x; q < 256; q += blockDim.x) pec[q] = A.pec[q];
}

__global__ void k_collect(KeyArgs A, uint32_t *table, int *overflow)
{
    __shared__ uint8_t pec[256];
    __shared__ uint32_t seen[kCache];   // keys this block has already put into the set
    __shared__ unsigned useen[8];       // the same for uniform keys (four equal ids), by id
    load_pec(A, pec);
    for (int q = threadIdx.x; q < kCache; q += blockDim.x) seen[q] = kEmpty;
    if (threadIdx.x < 8) useen[threadIdx.x] = 0u;
    __syncthreads();
    for (int k = blockIdx.z; k <= A.nz; k += gridDim.z)
        for (int j = blockIdx.y; j <= A.ny; j += gridDim.y)
        for (int i = threadIdx.x; i <= A.nx; i += blockDim.x) {
            const NodeCells n = node_cells(A, i, j, k);
            for (int comp = 0; comp < 3; ++comp) {
                uint32_t id[4];
                if (!edge_ids(A, n, comp, i, j, k, id)) continue;
                const bool uni = uniform(id);
                if (uni && (useen[id[0] >> 5] >> (id[0] & 31) & 1u)) continue;
                const uint32_t key = key_of(A, pec, id);
                if (key == kEmpty) continue;
                // a handful of distinct keys among millions of edges: after its first
                // insertion a key is found in the block's cache; the set's slot is read
                // before any compare-and-swap, so racing first insertions stay cheap
                const int c = (key * 2654435761u) >> (32 - 6);
                if (seen[c] == key) continue;
                uint32_t s = hash_slot(key);
                for (int probes = 0;; ++probes) {
                    if (probes >= kHashSize) { atomicOr(overflow, 1); break; }
                    const uint32_t cur = *(volatile const uint32_t *)&table[s];
                    if (cur == key) break;
                    if (cur == kEmpty) {
                        const uint32_t prev = atomicCAS(&table[s], kEmpty, key);
                        if (prev == kEmpty || prev == key) break;
                    }
                    s = (s + 1) & (kHashSize - 1);
                }
                if (uni) atomicOr(&useen[id[0] >> 5], 1u << (id[0] & 31));
                else seen[c] = key;
            }
        }
}

// uni_class[m]: class of an edge whose four cells are all material m (0 for PEC or absent)
__global__ void k_assign(KeyArgs A, const uint32_t *__restrict__ table, const uint8_t *__restrict__ slot_class,
                         const uint8_t *__restrict__ uni_class, uint8_t *cx, uint8_t *cy, uint8_t *cz)
{
    __shared__ uint8_t pec[256], uni[256];
    for (int q = threadIdx.x; q < 256; q += blockDim.x) uni[q] = uni_class[q];
    // (class << 32) | key, one 64-bit word so that a reader never pairs a key with another's class
    __shared__ unsigned long long cache[kCache];
    load_pec(A, pec);
    for (int q = threadIdx.x; q < kCache; q += blockDim.x) cache[q] = kEmpty;
    __syncthreads();
    uint8_t *out[3] = {cx, cy, cz};
    for (int k = blockIdx.z; k <= A.nz; k += gridDim.z)
        for (int j = blockIdx.y; j <= A.ny; j += gridDim.y)
        for (int i = threadIdx.x; i < A.px; i += blockDim.x) {
            const long q = (long)k * A.plane + (long)j * A.px + i;
            const NodeCells n = i <= A.nx ? node_cells(A, i, j, k) : NodeCells{0, 0, 0, 0, 0, 0, 0};
            for (int comp = 0; comp < 3; ++comp) {
                uint8_t cl = 0;
                uint32_t id[4];
                const bool live = i <= A.nx && edge_ids(A, n, comp, i, j, k, id);
                const bool flat = live && uniform(id);
                if (flat) cl = uni[id[0]];
                const uint32_t key = (live && !flat) ? key_of(A, pec, id) : kEmpty;
                if (key != kEmpty) {
                    const int c = (key * 2654435761u) >> (32 - 6);
                    const unsigned long long e = cache[c];
                    if ((uint32_t)e == key) {
                        cl = (uint8_t)(e >> 32);
                    } else {
                        uint32_t s = hash_slot(key);
                        for (int probes = 0; probes < kHashSize; ++probes) {
                            const uint32_t t = __ldg(&table[s]);
                            if (t == key) { cl = __ldg(&slot_class[s]); break; }
                            if (t == kEmpty) break;
                            s = (s + 1) & (kHashSize - 1);
                        }
                        cache[c] = ((unsigned long long)cl << 32) | key;
                    }
                }
                out[comp][q] = cl;
            }
        }
}

// zero-thickness sheet: class 0 on the in-plane edges (see yf_add_pec_sheet)
__global__ void k_sheet(uint8_t *ca, uint8_t *cb, int px, long plane, int ax, int idx, int lo0,
                        int hi0, int lo1, int hi1)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x;   // along axis 0 of the sheet
    const int v = blockIdx.y * blockDim.y + threadIdx.y;   // along axis 1
    if (lo0 + u > hi0 || lo1 + v > hi1) return;
    const int a = lo0 + u, b = lo1 + v;
    // edges along the first in-plane axis: a in [lo0, hi0), b in [lo1, hi1]
    // edges along the second in-plane axis: a in [lo0, hi0], b in [lo1, hi1)
    long q;
    if (ax == 2) q = (long)idx * plane + (long)b * px + a;      // (x, y) = (a, b), z = idx
    else if (ax == 1) q = (long)b * plane + (long)idx * px + a; // (x, z) = (a, b), y = idx
    else q = (long)b * plane + (long)a * px + idx;              // (y, z) = (a, b), x = idx
    if (a < hi0) ca[q] = 0;
    if (b < hi1) cb[q] = 0;
}

}  // namespace

yf_status derive_edge_classes(int nx, int ny, int nz, int px, long plane, const uint8_t *ids_dev,
                              int nmat, const double *eps_r, const double *sigma,
                              const uint8_t *is_pec, uint8_t *cls_dev[3], MaterialResult *res,
                              MatScratch *scratch, cudaStream_t s)
{
    uint8_t pec_h[256];
    memset(pec_h, 0, sizeof(pec_h));
    for (int m = 0; m < nmat; ++m) pec_h[m] = is_pec ? (is_pec[m] ? 1 : 0) : 0;

    std::vector<uint8_t> uni_h(256, 0);
    yf_status st = YF_OK;
    std::vector<uint32_t> keys(kHashSize);
    std::vector<uint8_t> slot_h(kHashSize, 0);
    KeyArgs A;
    int ovf = 0;
    const dim3 blk(256), grd(1, std::min(ny + 1, 128), std::min(nz + 1, 8));
    if (!scratch->table &&
        (cudaMalloc(&scratch->table, kHashSize * sizeof(uint32_t)) != cudaSuccess ||
         cudaMalloc(&scratch->slot_class, kHashSize) != cudaSuccess || cudaMalloc(&scratch->pec, 256) != cudaSuccess ||
         cudaMalloc(&scratch->uni, 256) != cudaSuccess ||
         cudaMalloc(&scratch->overflow, sizeof(int)) != cudaSuccess)) {
        mat_scratch_free(scratch);
        return fail(YF_E_OOM, "derive_edge_classes: device allocation failed");
    }
    uint32_t *const table = scratch->table;
    uint8_t *const slot_class = scratch->slot_class, *const pec_d = scratch->pec, *const uni_d = scratch->uni;
    int *const overflow = scratch->overflow;
    if (cudaMemsetAsync(table, 0xFF, kHashSize * sizeof(uint32_t), s) != cudaSuccess ||
        cudaMemsetAsync(overflow, 0, sizeof(int), s) != cudaSuccess ||
        cudaMemcpyAsync(pec_d, pec_h, 256, cudaMemcpyHostToDevice, s) != cudaSuccess) {
        st = fail(YF_E_CUDA, "derive_edge_classes: set-up copy failed");
        goto done;
    }
    A.ids = ids_dev; A.pec = pec_d; A.nmat = nmat; A.overflow = overflow; A.nx = nx; A.ny = ny; A.nz = nz; A.px = px; A.plane = plane;
    k_collect<<<grd, blk, 0, s>>>(A, table, overflow);
    if (cudaMemcpyAsync(keys.data(), table, kHashSize * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                        s) != cudaSuccess ||
        cudaMemcpyAsync(&ovf, overflow, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        st = fail(YF_E_CUDA, "derive_edge_classes: collecting keys failed: %s",
                  cudaGetErrorString(cudaGetLastError()));
        goto done;
    }
    if (ovf & 2) {
        st = fail(YF_E_INVALID, "material index >= nmat (%d) in ids", nmat);
        goto done;
    }
    if (ovf & 1) {
        st = fail(YF_E_UNSUPPORTED, "more than %d distinct edge material combinations", kHashSize);
        goto done;
    }
    {
        // (eps_r, sigma) of each key: mean over the four ids (sorted order)
        std::map<std::pair<double, double>, int> uniq;
        std::vector<std::pair<int, std::pair<double, double>>> slot_val;
        for (int sl = 0; sl < kHashSize; ++sl) {
            const uint32_t key = keys[sl];
            if (key == kEmpty) continue;
            double er = 0.0, sg = 0.0;
            for (int q = 0; q < 4; ++q) {
                const int id = (key >> (8 * q)) & 0xFF;
                er += eps_r[id];
                sg += sigma[id];
            }
            const std::pair<double, double> v(er / 4.0, sg / 4.0);
            uniq[v] = 0;
            slot_val.push_back({sl, v});
        }
        if ((int)uniq.size() > kMaxClasses - 1) {
            st = fail(YF_E_UNSUPPORTED, "%zu distinct edge materials (at most %d)", uniq.size(),
                      kMaxClasses - 1);
            goto done;
        }
        res->eps_r.assign(1, 0.0);
        res->sigma.assign(1, 0.0);
        int next = 1;
        for (auto &kv : uniq) {
            kv.second = next++;
            res->eps_r.push_back(kv.first.first);
            res->sigma.push_back(kv.first.second);
        }
        res->nclass = next;
        for (auto &sv : slot_val) slot_h[sv.first] = (uint8_t)uniq[sv.second];
        for (int sl = 0; sl < kHashSize; ++sl) {
            const uint32_t key = keys[sl];
            const uint32_t m = key & 0xFF;
            if (key != kEmpty && key == m * 0x01010101u) uni_h[m] = slot_h[sl];
        }
    }
    if (cudaMemcpyAsync(slot_class, slot_h.data(), kHashSize, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(uni_d, uni_h.data(), 256, cudaMemcpyHostToDevice, s) != cudaSuccess) {
        st = fail(YF_E_CUDA, "derive_edge_classes: upload failed");
        goto done;
    }
    k_assign<<<grd, blk, 0, s>>>(A, table, slot_class, uni_d, cls_dev[0], cls_dev[1], cls_dev[2]);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
        st = fail(YF_E_CUDA, "derive_edge_classes: class assignment failed");
        goto done;
    }
done:
    return st;
}

void mat_scratch_free(MatScratch *m)
{
    cudaFree(m->table);
    cudaFree(m->slot_class);
    cudaFree(m->pec);
    cudaFree(m->uni);
    cudaFree(m->overflow);
    *m = MatScratch{};
}

yf_status apply_pec_sheet(int nx, int ny, int nz, int px, long plane, uint8_t *cls_dev[3],
                          const int sh[6], cudaStream_t s)
{
    (void)nx; (void)ny; (void)nz;
    const int ax = sh[0];
    // first / second in-plane axis component arrays
    uint8_t *ca = ax == 0 ? cls_dev[1] : cls_dev[0];
    uint8_t *cb = ax == 2 ? cls_dev[1] : cls_dev[2];
    const int n0 = sh[3] - sh[2] + 1, n1 = sh[5] - sh[4] + 1;
    dim3 blk(16, 16), grd((n0 + 15) / 16, (n1 + 15) / 16);
    k_sheet<<<grd, blk, 0, s>>>(ca, cb, px, plane, ax, sh[1], sh[2], sh[3], sh[4], sh[5]);
    YF_CUDA_TRY(cudaGetLastError());
    return YF_OK;
}

}  // namespace yf
