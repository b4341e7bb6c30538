// The single-grid handle (opaque to ABI users).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
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

    // two field buffers, each ex, ey, ez, hx, hy, hz at stride npts; buf[cur] is current.
    // The fused step reads buf[cur] and writes buf[cur ^ 1]; the reference kernels update
    // buf[cur] in place.
    void *buf[2] = {};
    int cur = 0;
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
    int variant = 2;              // 0: reference H and E, 1: fused step, 2: fused + TMA
    uint8_t *cls_base = nullptr;  // the three class arrays, contiguous
    CUtensorMap tmF[2];           // field buffers as 4-D tensors (variant 2)
    CUtensorMap tmC;              // edge classes as a 4-D tensor
    int tmap_tile_y = 0;          // tile the maps were encoded for (0: not encoded)
    yf::SideStream side = {};     // frame launches of variant 2 overlap the interior
    int tile_y = 8;               // fused: block rows (block is 32 x tile_y)
    int kseg = 16;                // fused: z-planes per block
    int chunk = 32;               // steps per captured graph (even)
    cudaGraphExec_t graph[2] = {};   // one per starting buffer parity
};

namespace yf {
yf_status finalize(yf_grid *g);
double courant_limit_dt(double dx, double dy, double dz);
// uniform-line two-port extraction from FP64 DFTs laid out as
// [port][Vre, Vim, Ire, Iim][nf] (yf_sparams.cu)
yf_status sparams_uniform(int nf, const double *freqs, const double *dfts, int dir1, double z_ref,
                          double *S_star, double *S, double *Zr, double *Zc, double *tau);
}  // namespace yf
