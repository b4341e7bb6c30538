// Internal types shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "yeefdtd.h"

namespace yf {

// CODATA 2018 vacuum constants (SI)
constexpr double kC0 = 299792458.0;
constexpr double kMu0 = 1.25663706212e-6;
constexpr double kEps0 = 8.8541878128e-12;

constexpr int kMaxClasses = 256;   // uint8 edge classes, class 0 = PEC
constexpr int kMaxPorts = 16;
constexpr int kMaxKseg = 64;      // z-planes per block of the fused steps
constexpr int kEpiThreads = 256;   // block size of the per-step port epilogue
constexpr int kEpiSegPoints = 1024; // points per epilogue work item
constexpr int kEnergyBlocks = 592; // 4 x 148 SMs: fixed partial count -> fixed sum order

// Records a message for yf_last_error() and returns the status.
yf_status fail(yf_status s, const char *fmt, ...);
yf_status cuda_fail(cudaError_t e, const char *what);

#define YF_CUDA_TRY(expr)                                                     \
    do {                                                                      \
        cudaError_t e__ = (expr);                                             \
        if (e__ != cudaSuccess) return ::yf::cuda_fail(e__, #expr);           \
    } while (0)

// One port as the epilogue kernel sees it.
struct PortDev {
    int plane, dir, j0, j1, k0, k1, kb, kt, m;
    int nfreq;
    int foff;          // offset of this port's frequencies in the concatenated lists
    double vscale;     // -(dy dz) / width
};

template <typename T>
struct Fields {
    T *c[6];           // ex, ey, ez, hx, hy, hz
};

// CPML data the stencil kernels need, per axis a (0 = x, 1 = y, 2 = z):
//   lo/hi  : absorbing slab present on the low / high face
//   prof   : six profiles of length N_a + 1: b_e, a_e, 1/kappa_e at integer nodes,
//            b_h, a_h, 1/kappa_h at half nodes (entry p is position p + 1/2)
//   psi[q] : auxiliaries of the slab, q = 0,1 for the two E components with a
//            derivative along a, q = 2,3 for the two H components (order below)
//     axis x: Ey(dHz/dx), Ez(dHy/dx) | Hy(dEz/dx), Hz(dEy/dx)
//     axis y: Ex(dHz/dy), Ez(dHx/dy) | Hx(dEz/dy), Hz(dEx/dy)
//     axis z: Ex(dHy/dz), Ey(dHx/dz) | Hx(dEy/dz), Hy(dEx/dz)
//   slab index of position p: p (p < n) or n + p - (N - n) (p >= N - n); length 2n+1
//   psi layout: axis x [(k(ny+1) + j) L + s], axis y [(k L + s) px + i],
//               axis z [(s(ny+1) + j) px + i]
template <typename T>
struct Pml {
    int n;
    int lo[3], hi[3];
    int len;
    const T *prof[3];
    T *psi[3][4];
};

template <typename T>
struct StencilParams {
    int nx, ny, nz, px;
    long plane;        // px * (ny + 1)
    T rdx, rdy, rdz;   // 1 / d
    T db;              // dt / mu0
    const uint8_t *cls[3];
    const T *ctab;     // [kMaxClasses][2] = (Ca, Cb)
    Pml<T> pml;
};

template <typename T>
struct FusedArgs {
    int nx, ny, nz, px, kseg;
    int tx0, ty0;            // first tile of this launch (tile units)
    int z0, z1;              // planes z0..z1 of this launch
    long plane, npts;
    T rdx, rdy, rdz, db;
    const uint8_t *cls[3];
    const T *ctab;
    const T *A;              // old buffer: 6 components at stride npts
    T *B;                    // new buffer
    int n, L, lo[3], hi[3];  // CPML: thickness, slab length 2n+1, faces
    const T *prof[3];
    T *psiE[3][2];           // E auxiliaries (in place)
    const T *psiHr[3][2];    // H auxiliaries, read copy
    T *psiHw[3][2];          // H auxiliaries, write copy
};

// Work item of the port epilogue: kind 0 adds the source on points [start, start+count)
// of the source rectangle, kind 1 sums that range of a port's V surface, kind 2 of its
// I loops; kinds 1 and 2 leave their partial sum in slot[segment].
struct EpiSeg {
    int kind, port, start, count;
};

template <typename T>
struct EpiParams {
    const EpiSeg *segs;
    int nseg;
    double *slots;            // one partial per segment
    unsigned int *ticket;     // arrival counter of the blocks (reset by the last one)
    T *ez;                   // field buffer the source writes into and V reads
    const T *hy, *hz;        // H^{n+1/2}
    const uint8_t *cls_z;
    int nx, ny, nz, px;
    long plane;
    // source
    int src_kind, src_plane, sj0, sj1, sk0, sk1;
    double amp, p0, p1, t0, dt;
    const double *table;
    long table_len;
    // ports and DFT
    int nports;
    const PortDev *ports;
    const unsigned long long *inc;   // per frequency: round(f dt / 2 * 2^64)
    int dft_mask;
    double *acc64;   // [nf_total][4]  V re, V im, I re, I im
    float *acc32;    // [nf_total][4]
    float *kahan;    // [nf_total][8]  (sum, compensation) x 4
    double dy, dz;
    long long *ctr;      // steps whose ports and transforms are done
    long long *src_ctr;  // steps whose source is added (equal to *ctr between calls)
    int skip_source;     // 1: the source is added by k_epi_source on the critical path
    int *status;         // bit 0: non-finite port sample
};

// kernel launchers (yf_kernels.cu)
template <typename T>
cudaError_t launch_update_h(const StencilParams<T> &p, const Fields<T> &f, cudaStream_t s);
template <typename T>
cudaError_t launch_update_e(const StencilParams<T> &p, const Fields<T> &f, cudaStream_t s);
template <typename T>
cudaError_t launch_epilogue(const EpiParams<T> &p, cudaStream_t s);
// the soft source alone (one block; step index and counter *p.src_ctr)
template <typename T>
cudaError_t launch_epi_source(const EpiParams<T> &p, cudaStream_t s);
// one block per grid; grid q takes eps[stride q + parity]: stride 2 holds two parameter sets
// (buffer parity 0, 1) per grid, stride 3 one per buffer of three
template <typename T>
cudaError_t launch_epilogue_batch(const EpiParams<T> *eps, int n, int parity, cudaStream_t s, int stride = 2);
template <typename T>
cudaError_t launch_fused(const FusedArgs<T> &a, int tile_y, cudaStream_t s);
// TMA-staged fused step (yf_tma.cu); tmF maps buffer A as [6][nz+1][ny+1][px] with box
// (tma_box_x, tile_y + 2, 1, 3); tmC maps the classes [3][nz+1][ny+1][px] with box
// (32, tile_y, 1, 3)
template <typename T>
int tma_box_x(int tile_x);
cudaError_t tma_prepare();
// streams of a grid for work that may overlap the main stream within a step: one per CPML
// work kind, forked from and joined back into the main stream (graph capture turns them into
// parallel branches)
constexpr int kSideStreams = 4;
struct SideStream {
    cudaStream_t stream[kSideStreams];
    cudaEvent_t fork, join[kSideStreams];
    bool ready;
};
cudaError_t side_create(SideStream *s);
void side_destroy(SideStream *s);
// one block of the TMA-staged step: instance, tile origin (node indices), planes kb..ke
struct BatchItem {
    int inst, i0, j0, kb, ke;
};
// device-side plan of the TMA-staged step for one or many grids: work items grouped by kind
// (0 no CPML, 1 x CPML, 2 y CPML, 3 z CPML, 4 all), per-grid arguments for both buffer
// parities and per-grid tensor maps [grid][parity][field map, class map]
struct TmaPlan {
    BatchItem *items;
    int offset[5], count[5];
    void *args;
    CUtensorMap *maps;
    // argument sets per grid: 2 (two buffers, by parity) or 6 (three, by 2 * source + hpar);
    // 0 reads as 2.  Grid q's set p is args[stride q + p], its maps maps[2 (stride q + p) ..]
    int stride;
};
template <typename T>
cudaError_t launch_tma_plan(const TmaPlan &pl, int tile_y, int parity, int *status, cudaStream_t s,
                            const SideStream *side);
// mixed_seg > 0: the all-CPML kind (4) in segments of at most mixed_seg planes
void tma_items(int inst, int nx, int ny, int nz, int kseg, int tile_y, int n, const int lo[3],
               const int hi[3], std::vector<BatchItem> items[5], int mixed_seg = 0);
// two-step update of the inner box (yf_tb.cu, FP32): A = the buffer at step n (read through
// the tensor maps), C receives E^{n+2}, H^{n+3/2} on the box, B the box's outer node layer at
// E^{n+1}, H^{n+1/2}.  The box [bx0, bx1] x [by0, by1] x [bz0, bz1] is a union of 32 x 8 tiles.
// tile and TMA boxes of the two-step kernel
// output tile 32 x ty (ty = 8 or 16); E windows 40 x (ty + 4) nodes from (i0-4, j0-2), H windows
// 40 x (ty + 3) from the same corner, class tiles 80 x (ty + 2) bytes from (i0-16, j0-1)
constexpr int kTbTileX = 32;
constexpr int kTbWinX = 40;
constexpr int kTbClsX = 80;
struct TbArgs {
    int px;
    long plane, npts;
    float rdx, rdy, rdz, db;
    const float *ctab;
    float *B, *C;
    int bx0, bx1, by0, by1, bz0, bz1;
};
// plan of variant 4 for one grid
struct TbPlan {
    TmaPlan full;        // single step over the grid; arguments and maps by slot 2 * src + hpar
    TmaPlan frame;       // single step outside the box; shares full's arguments and maps
    BatchItem *items;    // two-step items of the box
    int count;
    TbArgs *args;        // [3] by source buffer
    CUtensorMap *maps;   // [3][window map, class map]
    int box[6];          // bx0, bx1, by0, by1, bz0, bz1
    int ty;              // tile height of the two-step blocks (8 or 16)
    cudaStream_t stream;
    cudaEvent_t fork, join;
    // recorded by a pair before its last epilogue: the next pair's box kernel waits on it (it
    // touches none of the nodes that epilogue reads or writes); valid while `chained`
    cudaEvent_t fork_next;
    bool chained;
    // the port integrals and running transforms of each step run on pstream, off the
    // critical path: ev_src (main stream, after a step's source) starts them; the next pair's
    // box kernel waits for ev_p1 (after the first step's), and the frame step of the pair
    // after it for ev_p2[parity] (after the second step's), before overwriting what they read
    cudaStream_t pstream;
    cudaEvent_t ev_src, ev_p1, ev_p2[2];
    int npair;           // pairs issued since the last join
};
cudaError_t tb_prepare();
cudaError_t launch_tb2(const BatchItem *items, int count, const TbArgs *args, const CUtensorMap *maps,
                       int phase, int *status, cudaStream_t s, int tile_y);
// skewed TMA-staged fused step (yf_skew.cu), same tensor maps as launch_tma
cudaError_t skew_prepare();
template <typename T>
cudaError_t launch_skew(const FusedArgs<T> &a, const CUtensorMap &tmF, const CUtensorMap &tmC,
                        int tile_y, int *status, cudaStream_t s);
template <typename T>
cudaError_t launch_sanitize(const Fields<T> &f, uint8_t *const cls[3], int nx, int ny, int nz,
                            int px, long plane, cudaStream_t s);
template <typename T>
cudaError_t launch_energy(const T *const c[6], const uint8_t *const cls[3], const double *eps_tab,
                          int nx, int ny, int nz, int px, long plane, double *partials,
                          double *out, cudaStream_t s);

// materials (yf_materials.cu)
struct MaterialResult {
    int nclass;                       // including class 0
    std::vector<double> eps_r, sigma; // per class (class 0 unused)
};
// device scratch of the class derivation, allocated on first use and kept by its owner
struct MatScratch {
    uint32_t *table = nullptr;
    uint8_t *slot_class = nullptr, *pec = nullptr, *uni = nullptr;
    int *overflow = nullptr;
};
void mat_scratch_free(MatScratch *m);
yf_status derive_edge_classes(int nx, int ny, int nz, int px, long plane, const uint8_t *ids_dev,
                              int nmat, const double *eps_r, const double *sigma,
                              const uint8_t *is_pec, uint8_t *cls_dev[3], MaterialResult *res,
                              MatScratch *scratch, cudaStream_t s);
yf_status apply_pec_sheet(int nx, int ny, int nz, int px, long plane, uint8_t *cls_dev[3],
                          const int sheet[6], cudaStream_t s);

}  // namespace yf
