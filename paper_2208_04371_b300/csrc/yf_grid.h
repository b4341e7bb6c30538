// The single-grid handle (opaque to ABI users).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "yf_internal.h"

struct yf_grid {
    // geometry: fields are (nz+1) planes of (ny+1) rows of px elements, x fastest
    int nx = 0, ny = 0, nz = 0, px = 0;
    long plane = 0, npts = 0;
    double dx = 0, dy = 0, dz = 0, dt = 0;
    yf_prec prec = YF_FP32;
    size_t esz = 4;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // host ids cross and their classes are derived on mstream, beside the zeroing that
    // yf_reset queues on `stream`; `stream` then waits for mat_ready (created on first use)
    cudaStream_t mstream = nullptr;
    cudaEvent_t mat_ready = nullptr;

    // field buffers, each ex, ey, ez, hx, hy, hz at stride npts; buf[cur] is current.
    // The fused step reads buf[cur] and writes the next buffer (buf[cur ^ 1]; variant 4
    // rotates three: buf[(cur + 1) % 3]); the reference kernels update buf[cur] in place.
    // buf[2] exists only while variant 4 is set.
    void *buf[3] = {};
    int cur = 0;
    int next_buf(int b) const { return buf[2] ? (b + 1) % 3 : b ^ 1; }
    int nbuf() const { return buf[2] ? 3 : 2; }
    void *fld(int c) const { return (char *)buf[cur] + (size_t)c * npts * esz; }
    uint8_t *cls[3] = {};         // per-edge material class of ex, ey, ez (0 = PEC)
    void *ctab = nullptr;         // [256][2] (Ca, Cb) in field precision
    double *eps_tab = nullptr;    // [256] eps0 eps_r per class
    yf::MaterialResult mat;
    bool materials_done = false;
    std::vector<int> sheets;      // 6 ints per sheet

    int bc[6] = {};
    int pml_n = 8, pml_order = 3;
    double pml_sigma_scale = 1.0, pml_kappa_max = 1.0, pml_alpha_max = 0.0;
    int pml_lo[3] = {}, pml_hi[3] = {};
    void *prof[3] = {};
    // CPML auxiliaries per axis: psiE[a][0..1] (E, updated in place) and two copies of the
    // H ones, psiH[par][a][0..1]; psiH[hpar] is current (see Pml in yf_internal.h for order)
    void *psiE[3][2] = {};
    void *psiH[2][3][2] = {};
    int hpar = 0;
    size_t psi_count[3] = {};

    bool has_src = false;
    yf_waveform src = {};
    int src_plane = 0, sj0 = 0, sj1 = 0, sk0 = 0, sk1 = 0;
    std::vector<double> src_table_host;
    double *src_table_dev = nullptr;
    long src_table_len = 0;

    std::vector<yf::PortDev> ports;
    std::vector<double> freqs;                // concatenated per-port lists
    std::vector<unsigned long long> inc;      // concatenated phase increments
    int nf_total = 0;
    yf::PortDev *ports_dev = nullptr;
    unsigned long long *inc_dev = nullptr;
    double *acc64 = nullptr;
    float *acc32 = nullptr, *kahan = nullptr;
    int dft_mask = YF_DFT_FP64;
    std::vector<yf::EpiSeg> segs;
    yf::EpiSeg *segs_dev = nullptr;
    double *slots = nullptr;
    unsigned int *ticket = nullptr;

    long long *ctr = nullptr;     // device: steps completed
    int *status = nullptr;        // device: error bits
    long steps_done = 0;
    double *energy_partials = nullptr;   // scratch of the energy reduction (+1 result slot)

    bool started = false;
    bool geometry_open = false;   // after yf_reset: materials and sheets may change
    int variant = 2;              // 0: reference H and E, 1: fused step, 2: fused + TMA,
                                  // 3: skewed, 4: two-step inner box (FP32)
    uint8_t *cls_base = nullptr;  // the three class arrays, contiguous
    CUtensorMap tmF[3];           // field buffers as 4-D tensors (variants 2 to 4)
    CUtensorMap tmC;              // edge classes as a 4-D tensor
    int tmap_tile_y = 0;          // tile the maps were encoded for (0: not encoded)
    yf::SideStream side = {};     // CPML work of variant 2 overlaps the interior
    yf::TmaPlan plan = {};        // work items / arguments / maps of variant 2 (a batch of one)
    bool plan_ok = false;
    int tile_y = 8;               // fused: block rows (block is 32 x tile_y)
    int kseg = 16;                // fused: z-planes per block
    int box_seg = 0;              // variant 4: z-planes per two-step block (0: 2 kseg)
    int box_ty = 8;               // variant 4: tile height of the two-step blocks (8 or 16)
    int chunk = 32;               // steps per captured graph (even)
    cudaGraphExec_t graph[6] = {};   // one per starting state cur * 2 + hpar
    yf::TbPlan *tb = nullptr;        // variant 4
    yf::MatScratch mat_scratch;      // device scratch of the class derivation
    uint8_t *ids_stage = nullptr;    // host material ids staged on the device (re-solving grids)
};

namespace yf {
yf_status finalize(yf_grid *g);
yf_status encode_maps(yf_grid *g);
yf_status reset_state(yf_grid *g);
cudaError_t step_direct(yf_grid *g, cudaStream_t s);   // one un-graphed step
// autotuner cache (yf_tune.cu): "key": [tile_y, kseg, ms] entries in a small JSON object
bool tune_cache_get(const char *path, const std::string &key, int *tile_y, int *kseg);
void tune_cache_put(const char *path, const std::string &key, int tile_y, int kseg, double ms);
std::string tune_key(const char *kind, yf_prec prec, long cells, int pml);
// plan of the TMA-staged step over the given grids (yf_batch.cu); tensor maps must be encoded
// for tile_y
template <typename T>
yf_status build_plan(const std::vector<yf_grid *> &grids, int tile_y, int kseg, TmaPlan *pl);
void free_plan(TmaPlan *pl);
// variant 4 (yf_tb.cu): plan (box, work items, arguments, maps) for the current buffers;
// one time step over the whole grid; two time steps (box + frame); teardown
yf_status tb_build(yf_grid *g);
void tb_free(yf_grid *g);
cudaError_t tb_single(yf_grid *g, cudaStream_t s);
cudaError_t tb_pair(yf_grid *g, cudaStream_t s, const cudaEvent_t *ev = nullptr);
void tb_unchain(yf_grid *g);   // the next pair forks after everything queued before it
// main stream waits for the port epilogues still running on the side stream (ends a run of
// pairs; issued into the stream, so inside a capture too)
cudaError_t tb_join(yf_grid *g, cudaStream_t s);
int tb_launches_pair(const yf_grid *g);
int tb_launches_single(const yf_grid *g);
// the pieces of a variant-4 plan for one grid, shared with the batched two-step path
// (yf_tb_plan.cu): the inner box (false when none fits); the work items of grid `inst`
// (one-step over the grid, one-step outside the box, two-step box items of 32 x ty tiles and
// seg planes); the one-step arguments and maps by slot 2 * src + hpar; the two-step arguments
// and maps by source buffer
bool choose_box(const yf_grid *g, int box[6]);
void tb_items(const yf_grid *g, int inst, bool have_box, const int box[6], int ty, int seg,
              std::vector<BatchItem> full[5], std::vector<BatchItem> frame[5], std::vector<BatchItem> &two,
              int mixed_seg = 8);
void tb_step_args(yf_grid *g, FusedArgs<float> fa[6], CUtensorMap fm[12]);
yf_status tb_box_args(yf_grid *g, const int box[6], int ty, TbArgs ta[3], CUtensorMap tm[9]);
template <typename T>
Fields<T> fields_of(const yf_grid *g, int b);
template <typename T>
FusedArgs<T> fused_args(const yf_grid *g);   // A = buf[cur], psi H read = psiH[hpar]
template <typename T>
EpiParams<T> epi_params(const yf_grid *g);   // fields of buf[cur]
double courant_limit_dt(double dx, double dy, double dz);
// uniform-line two-port extraction from FP64 DFTs laid out as
// [port][Vre, Vim, Ire, Iim][nf] (yf_sparams.cu)
yf_status sparams_uniform(int nf, const double *freqs, const double *dfts, int dir1, double z_ref,
                          double *S_star, double *S, double *Zr, double *Zc, double *tau);
}  // namespace yf
