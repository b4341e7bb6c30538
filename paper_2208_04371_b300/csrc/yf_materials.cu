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

// key of edge `comp` at node (i, j, k); kEmpty for PEC / wall / non-existent edges
__device__ uint32_t edge_key(const KeyArgs &A, int comp, int i, int j, int k)
{
    int c[4][3];
    if (comp == 0) {            // E_x(i+1/2, j, k)
        if (i >= A.nx || j < 1 || j >= A.ny || k < 1 || k >= A.nz) return kEmpty;
        int t[4][3] = {{i, j - 1, k - 1}, {i, j, k - 1}, {i, j - 1, k}, {i, j, k}};
        memcpy(c, t, sizeof(c));
    } else if (comp == 1) {     // E_y(i, j+1/2, k)
        if (i < 1 || i >= A.nx || j >= A.ny || k < 1 || k >= A.nz) return kEmpty;
        int t[4][3] = {{i - 1, j, k - 1}, {i, j, k - 1}, {i - 1, j, k}, {i, j, k}};
        memcpy(c, t, sizeof(c));
    } else {                    // E_z(i, j, k+1/2)
        if (i < 1 || i >= A.nx || j < 1 || j >= A.ny || k >= A.nz) return kEmpty;
        int t[4][3] = {{i - 1, j - 1, k}, {i, j - 1, k}, {i - 1, j, k}, {i, j, k}};
        memcpy(c, t, sizeof(c));
    }
    uint32_t id[4];
    for (int q = 0; q < 4; ++q) {
        id[q] = A.ids[((long)c[q][2] * A.ny + c[q][1]) * A.nx + c[q][0]];
        if ((int)id[q] >= A.nmat) { atomicOr(A.overflow, 2); return kEmpty; }
        if (A.pec[id[q]]) return kEmpty;
    }
    cswap(id[0], id[1]); cswap(id[2], id[3]); cswap(id[0], id[2]); cswap(id[1], id[3]);
    cswap(id[1], id[2]);
    return id[0] | (id[1] << 8) | (id[2] << 16) | (id[3] << 24);
}

__device__ __forceinline__ uint32_t hash_slot(uint32_t key)
{
    return (key * 2654435761u) >> (32 - kHashBits);
}

__global__ void k_collect(KeyArgs A, uint32_t *table, int *overflow)
{
    const long npts = A.plane * (A.nz + 1);
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < npts;
         q += (long)gridDim.x * blockDim.x) {
        const int k = (int)(q / A.plane);
        const int r = (int)(q % A.plane);
        const int j = r / A.px, i = r % A.px;
        if (i > A.nx || j > A.ny) continue;
        for (int comp = 0; comp < 3; ++comp) {
            const uint32_t key = edge_key(A, comp, i, j, k);
            // a handful of distinct keys among millions of edges: one lane per distinct key
            // of the warp inserts, and a slot is read before any compare-and-swap, so the set
            // fills with a few atomics instead of one contended atomic per edge
            const unsigned active = __activemask();
            const unsigned peers = __match_any_sync(active, key);
            if (key == kEmpty || (int)(__ffs(peers) - 1) != (int)(threadIdx.x & 31)) continue;
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
        }
    }
}

__global__ void k_assign(KeyArgs A, const uint32_t *table, const uint8_t *slot_class,
                         uint8_t *cx, uint8_t *cy, uint8_t *cz)
{
    const long npts = A.plane * (A.nz + 1);
    uint8_t *out[3] = {cx, cy, cz};
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < npts;
         q += (long)gridDim.x * blockDim.x) {
        const int k = (int)(q / A.plane);
        const int r = (int)(q % A.plane);
        const int j = r / A.px, i = r % A.px;
        for (int comp = 0; comp < 3; ++comp) {
            uint8_t cl = 0;
            if (i <= A.nx && j <= A.ny) {
                const uint32_t key = edge_key(A, comp, i, j, k);
                if (key != kEmpty) {
                    uint32_t s = hash_slot(key);
                    for (int probes = 0; probes < kHashSize; ++probes) {
                        if (table[s] == key) { cl = slot_class[s]; break; }
                        if (table[s] == kEmpty) break;
                        s = (s + 1) & (kHashSize - 1);
                    }
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
                              cudaStream_t s)
{
    uint8_t pec_h[256];
    memset(pec_h, 0, sizeof(pec_h));
    for (int m = 0; m < nmat; ++m) pec_h[m] = is_pec ? (is_pec[m] ? 1 : 0) : 0;

    uint32_t *table = nullptr;
    uint8_t *slot_class = nullptr, *pec_d = nullptr;
    int *overflow = nullptr;
    yf_status st = YF_OK;
    std::vector<uint32_t> keys(kHashSize);
    std::vector<uint8_t> slot_h(kHashSize, 0);
    KeyArgs A;
    int ovf = 0;
    if (cudaMalloc(&table, kHashSize * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&slot_class, kHashSize) != cudaSuccess || cudaMalloc(&pec_d, 256) != cudaSuccess ||
        cudaMalloc(&overflow, sizeof(int)) != cudaSuccess) {
        st = fail(YF_E_OOM, "derive_edge_classes: device allocation failed");
        goto done;
    }
    if (cudaMemsetAsync(table, 0xFF, kHashSize * sizeof(uint32_t), s) != cudaSuccess ||
        cudaMemsetAsync(overflow, 0, sizeof(int), s) != cudaSuccess ||
        cudaMemcpyAsync(pec_d, pec_h, 256, cudaMemcpyHostToDevice, s) != cudaSuccess) {
        st = fail(YF_E_CUDA, "derive_edge_classes: set-up copy failed");
        goto done;
    }
    A.ids = ids_dev; A.pec = pec_d; A.nmat = nmat; A.overflow = overflow; A.nx = nx; A.ny = ny; A.nz = nz; A.px = px; A.plane = plane;
    k_collect<<<1184, 256, 0, s>>>(A, table, overflow);
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
    }
    if (cudaMemcpyAsync(slot_class, slot_h.data(), kHashSize, cudaMemcpyHostToDevice, s) !=
        cudaSuccess) {
        st = fail(YF_E_CUDA, "derive_edge_classes: upload failed");
        goto done;
    }
    k_assign<<<1184, 256, 0, s>>>(A, table, slot_class, cls_dev[0], cls_dev[1], cls_dev[2]);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
        st = fail(YF_E_CUDA, "derive_edge_classes: class assignment failed");
        goto done;
    }
done:
    if (table) cudaFree(table);
    if (slot_class) cudaFree(slot_class);
    if (pec_d) cudaFree(pec_d);
    if (overflow) cudaFree(overflow);
    return st;
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
