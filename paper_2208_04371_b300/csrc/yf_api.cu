// C ABI of the single-grid solver: handle life cycle, set-up, time stepping with captured
// CUDA graphs, read-out and checkpoints.  See include/yeefdtd.h for the contract.
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "yf_internal.h"
#include "yf_grid.h"

namespace yf {

static thread_local std::string g_err;

yf_status fail(yf_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

yf_status cuda_fail(cudaError_t e, const char *what)
{
    cudaGetLastError();   // clear a non-sticky error (e.g. a failed allocation) for later checks
    if (e == cudaErrorMemoryAllocation) return fail(YF_E_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(YF_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

double courant_limit_dt(double dx, double dy, double dz)
{
    return 1.0 / (kC0 * std::sqrt(1.0 / (dx * dx) + 1.0 / (dy * dy) + 1.0 / (dz * dz)));
}

// CPML profile at position pos (cells) along an axis of N cells; same grading as the
// absorbing-layer description in yf_set_pml.
static void pml_point(const yf_grid *g, int axis, int N, double delta, double pos, double *b,
                      double *a, double *rk)
{
    double depth = 0.0;
    const double L = (double)g->pml_n;
    if (g->pml_n > 0) {
        if (g->bc[2 * axis] == YF_BC_PML && pos < L) depth = (L - pos) / L;
        if (g->bc[2 * axis + 1] == YF_BC_PML && pos > N - L) depth = (pos - (N - L)) / L;
    }
    if (depth <= 0.0) {
        *b = 1.0; *a = 0.0; *rk = 1.0;
        return;
    }
    const double m = (double)g->pml_order;
    const double eta0 = std::sqrt(kMu0 / kEps0);
    const double smax = g->pml_sigma_scale * 0.8 * (m + 1.0) / (eta0 * delta);
    const double gr = std::pow(depth, m);
    const double sg = smax * gr;
    const double kap = 1.0 + (g->pml_kappa_max - 1.0) * gr;
    const double al = g->pml_alpha_max * (1.0 - depth);
    *b = std::exp(-(sg / kap + al) * g->dt / kEps0);
    *a = (sg > 0.0) ? sg / (sg * kap + kap * kap * al) * (*b - 1.0) : 0.0;
    *rk = 1.0 / kap;
}

template <typename T>
static yf_status upload_as(void **dst, const std::vector<double> &src)
{
    std::vector<T> tmp(src.begin(), src.end());
    YF_CUDA_TRY(cudaMalloc(dst, tmp.size() * sizeof(T)));
    YF_CUDA_TRY(cudaMemcpy(*dst, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice));
    return YF_OK;
}

static yf_status build_coeff_tables(yf_grid *g)
{
    std::vector<double> tab(2 * kMaxClasses, 0.0), eps(kMaxClasses, 0.0);
    for (int c = 1; c < g->mat.nclass; ++c) {
        const double e = kEps0 * g->mat.eps_r[c];
        const double loss = g->mat.sigma[c] * g->dt / (2.0 * e);
        tab[2 * c] = (1.0 - loss) / (1.0 + loss);
        tab[2 * c + 1] = (g->dt / e) / (1.0 + loss);
        eps[c] = e;
    }
    if (g->prec == YF_FP32) {
        std::vector<float> t32(tab.begin(), tab.end());
        YF_CUDA_TRY(cudaMemcpy(g->ctab, t32.data(), t32.size() * sizeof(float), cudaMemcpyHostToDevice));
    } else {
        YF_CUDA_TRY(cudaMemcpy(g->ctab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    YF_CUDA_TRY(cudaMemcpy(g->eps_tab, eps.data(), eps.size() * sizeof(double), cudaMemcpyHostToDevice));
    return YF_OK;
}

// the edge classes and their coefficient tables from device ids, on stream s (the grid's stream,
// or its materials stream for host ids); returns after s has finished
static yf_status derive_materials(yf_grid *g, const uint8_t *ids_dev, int nmat, const double *eps_r,
                                  const double *sigma, const uint8_t *is_pec, cudaStream_t s)
{
    yf_status st = derive_edge_classes(g->nx, g->ny, g->nz, g->px, g->plane, ids_dev, nmat, eps_r,
                                       sigma, is_pec, g->cls, &g->mat, &g->mat_scratch, s);
    if (st != YF_OK) return st;
    st = build_coeff_tables(g);
    if (st != YF_OK) return st;
    for (size_t q = 0; q < g->sheets.size(); q += 6) {
        st = apply_pec_sheet(g->nx, g->ny, g->nz, g->px, g->plane, g->cls, &g->sheets[q], s);
        if (st != YF_OK) return st;
    }
    YF_CUDA_TRY(cudaStreamSynchronize(s));
    g->materials_done = true;
    return YF_OK;
}

static yf_status build_pml(yf_grid *g)
{
    const int N[3] = {g->nx, g->ny, g->nz};
    const double D[3] = {g->dx, g->dy, g->dz};
    const int n = g->pml_n;
    for (int a = 0; a < 3; ++a) {
        g->pml_lo[a] = (n > 0 && g->bc[2 * a] == YF_BC_PML);
        g->pml_hi[a] = (n > 0 && g->bc[2 * a + 1] == YF_BC_PML);
        if (!g->pml_lo[a] && !g->pml_hi[a]) continue;
        if (N[a] < 2 * n + 1)
            return fail(YF_E_INVALID, "axis %d has %d cells, PML of %d cells needs >= %d", a, N[a], n,
                        2 * n + 1);
        const int N1 = N[a] + 1;
        std::vector<double> prof(6 * N1, 0.0);
        for (int p = 0; p <= N[a]; ++p)
            pml_point(g, a, N[a], D[a], (double)p, &prof[0 * N1 + p], &prof[1 * N1 + p], &prof[2 * N1 + p]);
        for (int p = 0; p < N[a]; ++p)
            pml_point(g, a, N[a], D[a], p + 0.5, &prof[3 * N1 + p], &prof[4 * N1 + p], &prof[5 * N1 + p]);
        yf_status st = g->prec == YF_FP32 ? upload_as<float>(&g->prof[a], prof)
                                          : upload_as<double>(&g->prof[a], prof);
        if (st != YF_OK) return st;
        const int L = 2 * n + 1;
        size_t cnt;
        if (a == 0) cnt = (size_t)(g->nz + 1) * (g->ny + 1) * L;
        else if (a == 1) cnt = (size_t)(g->nz + 1) * L * g->px;
        else cnt = (size_t)L * (g->ny + 1) * g->px;
        g->psi_count[a] = cnt;
        void **slots[6] = {&g->psiE[a][0], &g->psiE[a][1], &g->psiH[0][a][0], &g->psiH[0][a][1],
                           &g->psiH[1][a][0], &g->psiH[1][a][1]};
        for (int q = 0; q < 6; ++q) {
            YF_CUDA_TRY(cudaMalloc(slots[q], cnt * g->esz));
            YF_CUDA_TRY(cudaMemset(*slots[q], 0, cnt * g->esz));
        }
    }
    return YF_OK;
}

// tensor maps of the TMA-staged step, for the grid's current tile height
yf_status encode_maps(yf_grid *g)
{
    if (g->tmap_tile_y == g->tile_y) return YF_OK;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                         cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return fail(YF_E_CUDA, "cuTensorMapEncodeTiled is not available");
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    const int esz = (int)g->esz;
    const int bx = esz == 4 ? tma_box_x<float>(32) : tma_box_x<double>(32);
    const cuuint64_t gdim[4] = {(cuuint64_t)g->px, (cuuint64_t)(g->ny + 1), (cuuint64_t)(g->nz + 1), 6};
    const cuuint64_t gstr[3] = {(cuuint64_t)g->px * esz, (cuuint64_t)g->plane * esz,
                                (cuuint64_t)g->npts * esz};
    const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)(g->tile_y + 2), 1, 3};
    // 64-byte L2 promotion: a window row (160 bytes from 16 bytes before the tile) would pull
    // three 128-byte lines from DRAM at a tile whose neighbours run in another launch (the
    // CPML frame)
    const cuuint32_t one[4] = {1, 1, 1, 1};
    for (int b = 0; b < g->nbuf(); ++b) {
        CUresult r = encode(&g->tmF[b], esz == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                            4, g->buf[b], gdim, gstr, box, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_64B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(YF_E_CUDA, "encoding the field tensor map failed (%d)", (int)r);
    }
    const cuuint64_t cdim[4] = {(cuuint64_t)g->px, (cuuint64_t)(g->ny + 1), (cuuint64_t)(g->nz + 1), 3};
    const cuuint64_t cstr[3] = {(cuuint64_t)g->px, (cuuint64_t)g->plane, (cuuint64_t)g->npts};
    const cuuint32_t cbox[4] = {32, (cuuint32_t)g->tile_y, 1, 3};
    CUresult r = encode(&g->tmC, CU_TENSOR_MAP_DATA_TYPE_UINT8, 4, g->cls_base, cdim, cstr, cbox, one,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_64B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(YF_E_CUDA, "encoding the class tensor map failed (%d)", (int)r);
    YF_CUDA_TRY(tma_prepare());
    YF_CUDA_TRY(skew_prepare());
    g->tmap_tile_y = g->tile_y;
    return YF_OK;
}

static yf_status ensure_plan(yf_grid *g)
{
    if (g->plan_ok) return YF_OK;
    yf_status st = encode_maps(g);
    if (st != YF_OK) return st;
    std::vector<yf_grid *> one(1, g);
    st = g->prec == YF_FP32 ? build_plan<float>(one, g->tile_y, g->kseg, &g->plan)
                            : build_plan<double>(one, g->tile_y, g->kseg, &g->plan);
    if (st != YF_OK) return st;
    g->plan_ok = true;
    return YF_OK;
}

template <typename T>
Fields<T> fields_of(const yf_grid *g, int b)
{
    Fields<T> F;
    for (int c = 0; c < 6; ++c) F.c[c] = (T *)((char *)g->buf[b] + (size_t)c * g->npts * g->esz);
    return F;
}

template <typename T>
StencilParams<T> stencil_params(const yf_grid *g)
{
    StencilParams<T> P;
    P.nx = g->nx; P.ny = g->ny; P.nz = g->nz; P.px = g->px; P.plane = g->plane;
    P.rdx = (T)(1.0 / g->dx); P.rdy = (T)(1.0 / g->dy); P.rdz = (T)(1.0 / g->dz);
    P.db = (T)(g->dt / kMu0);
    for (int c = 0; c < 3; ++c) P.cls[c] = g->cls[c];
    P.ctab = (const T *)g->ctab;
    P.pml.n = g->pml_n;
    P.pml.len = 2 * g->pml_n + 1;
    for (int a = 0; a < 3; ++a) {
        P.pml.lo[a] = g->pml_lo[a];
        P.pml.hi[a] = g->pml_hi[a];
        P.pml.prof[a] = (const T *)g->prof[a];
        P.pml.psi[a][0] = (T *)g->psiE[a][0];
        P.pml.psi[a][1] = (T *)g->psiE[a][1];
        P.pml.psi[a][2] = (T *)g->psiH[g->hpar][a][0];
        P.pml.psi[a][3] = (T *)g->psiH[g->hpar][a][1];
    }
    return P;
}

template <typename T>
FusedArgs<T> fused_args(const yf_grid *g)
{
    FusedArgs<T> F;
    F.nx = g->nx; F.ny = g->ny; F.nz = g->nz; F.px = g->px; F.kseg = g->kseg;
    F.tx0 = 0; F.ty0 = 0; F.z0 = 0; F.z1 = g->nz;
    F.plane = g->plane; F.npts = g->npts;
    F.rdx = (T)(1.0 / g->dx); F.rdy = (T)(1.0 / g->dy); F.rdz = (T)(1.0 / g->dz);
    F.db = (T)(g->dt / kMu0);
    for (int c = 0; c < 3; ++c) F.cls[c] = g->cls[c];
    F.ctab = (const T *)g->ctab;
    F.A = (const T *)g->buf[g->cur];
    F.B = (T *)g->buf[g->next_buf(g->cur)];
    F.n = g->pml_n;
    F.L = 2 * g->pml_n + 1;
    for (int a = 0; a < 3; ++a) {
        F.lo[a] = g->pml_lo[a];
        F.hi[a] = g->pml_hi[a];
        F.prof[a] = (const T *)g->prof[a];
        for (int q = 0; q < 2; ++q) {
            F.psiE[a][q] = (T *)g->psiE[a][q];
            F.psiHr[a][q] = (const T *)g->psiH[g->hpar][a][q];
            F.psiHw[a][q] = (T *)g->psiH[g->hpar ^ 1][a][q];
        }
    }
    return F;
}

template <typename T>
EpiParams<T> epi_params(const yf_grid *g)
{
    EpiParams<T> E;
    E.segs = g->segs_dev; E.nseg = (int)g->segs.size(); E.slots = g->slots; E.ticket = g->ticket;
    E.ez = (T *)g->fld(2); E.hy = (const T *)g->fld(4); E.hz = (const T *)g->fld(5);
    E.cls_z = g->cls[2];
    E.nx = g->nx; E.ny = g->ny; E.nz = g->nz; E.px = g->px; E.plane = g->plane;
    E.src_kind = g->has_src ? g->src.kind : YF_WAVE_NONE;
    E.src_plane = g->src_plane; E.sj0 = g->sj0; E.sj1 = g->sj1; E.sk0 = g->sk0; E.sk1 = g->sk1;
    E.amp = g->src.amplitude; E.p0 = g->src.p0; E.p1 = g->src.p1; E.t0 = g->src.t0; E.dt = g->dt;
    E.table = g->src_table_dev; E.table_len = g->src_table_len;
    E.nports = (int)g->ports.size();
    E.ports = g->ports_dev; E.inc = g->inc_dev; E.dft_mask = g->dft_mask;
    E.acc64 = g->acc64; E.acc32 = g->acc32; E.kahan = g->kahan;
    E.dy = g->dy; E.dz = g->dz;
    E.ctr = g->ctr; E.src_ctr = g->ctr + 1; E.skip_source = 0; E.status = g->status;
    return E;
}

template Fields<float> fields_of<float>(const yf_grid *, int);
template Fields<double> fields_of<double>(const yf_grid *, int);
template FusedArgs<float> fused_args<float>(const yf_grid *);
template FusedArgs<double> fused_args<double>(const yf_grid *);
template EpiParams<float> epi_params<float>(const yf_grid *);
template EpiParams<double> epi_params<double>(const yf_grid *);

// epilogue work items: source rectangle, each port's V surface and I loops
static void build_segments(yf_grid *g)
{
    g->segs.clear();
    auto add = [&](int kind, int port, int total) {
        for (int s = 0; s < total; s += kEpiSegPoints)
            g->segs.push_back({kind, port, s, total - s < kEpiSegPoints ? total - s : kEpiSegPoints});
    };
    if (g->has_src) add(0, -1, (g->sj1 - g->sj0 + 1) * (g->sk1 - g->sk0));
    for (int p = 0; p < (int)g->ports.size(); ++p) {
        const PortDev &d = g->ports[p];
        add(1, p, (d.j1 - d.j0 + 1) * (d.k1 - d.k0));
        const int nyl = d.j1 - d.j0 + 2 * d.m - 1, nzl = d.kt - d.kb + 2 * d.m - 1;
        add(2, p, 2 * (2 * nyl + 2 * nzl));
    }
}

// variant 4: a third field buffer equal to the current one (nodes no kernel writes must agree
// in all buffers), maps for it, and the plan
static yf_status enter_tb(yf_grid *g)
{
    if (g->prec != YF_FP32) return fail(YF_E_INVALID, "variant 4 needs FP32 fields");
    const size_t bytes = 6 * g->npts * g->esz;
    YF_CUDA_TRY(cudaStreamSynchronize(g->stream));
    if (!g->buf[2]) {
        YF_CUDA_TRY(cudaMalloc(&g->buf[2], bytes));
        g->tmap_tile_y = 0;
    }
    for (int b = 0; b < 3; ++b)
        if (b != g->cur) YF_CUDA_TRY(cudaMemcpy(g->buf[b], g->buf[g->cur], bytes, cudaMemcpyDeviceToDevice));
    yf_status st = encode_maps(g);
    if (st != YF_OK) return st;
    return tb_build(g);
}

// back to two buffers: the current fields move to buf[0] or stay in buf[1]; the auxiliary
// copies are relabelled so that hpar == cur again (the two-buffer plans assume it)
static yf_status leave_tb(yf_grid *g)
{
    tb_free(g);
    if (!g->buf[2]) return YF_OK;
    YF_CUDA_TRY(cudaStreamSynchronize(g->stream));
    const size_t bytes = 6 * g->npts * g->esz;
    if (g->cur == 2) {
        YF_CUDA_TRY(cudaMemcpy(g->buf[0], g->buf[2], bytes, cudaMemcpyDeviceToDevice));
        g->cur = 0;
    }
    YF_CUDA_TRY(cudaMemcpy(g->buf[g->cur ^ 1], g->buf[g->cur], bytes, cudaMemcpyDeviceToDevice));
    cudaFree(g->buf[2]);
    g->buf[2] = nullptr;
    if (g->hpar != g->cur) {
        for (int a = 0; a < 3; ++a)
            for (int q = 0; q < 2; ++q) std::swap(g->psiH[0][a][q], g->psiH[1][a][q]);
        g->hpar = g->cur;
    }
    g->tmap_tile_y = 0;
    return YF_OK;
}

yf_status finalize(yf_grid *g)
{
    if (g->started) return YF_OK;
    yf_status st;
    if (!g->materials_done) {
        uint8_t *ids = nullptr;
        const size_t ncell = (size_t)g->nx * g->ny * g->nz;
        YF_CUDA_TRY(cudaMalloc(&ids, ncell));
        YF_CUDA_TRY(cudaMemset(ids, 0, ncell));
        const double er = 1.0, sg = 0.0;
        const uint8_t pec = 0;
        st = derive_materials(g, ids, 1, &er, &sg, &pec, g->stream);
        cudaFree(ids);
        if (st != YF_OK) return st;
    }
    st = build_pml(g);
    if (st != YF_OK) return st;
    // ports and DFT accumulators
    const int np = (int)g->ports.size();
    int total = 0;
    for (int p = 0; p < np; ++p) total += g->ports[p].nfreq;
    g->nf_total = total;
    if (np > 0) {
        YF_CUDA_TRY(cudaMalloc(&g->ports_dev, np * sizeof(PortDev)));
        YF_CUDA_TRY(cudaMemcpy(g->ports_dev, g->ports.data(), np * sizeof(PortDev), cudaMemcpyHostToDevice));
        YF_CUDA_TRY(cudaMalloc(&g->inc_dev, total * sizeof(unsigned long long)));
        YF_CUDA_TRY(cudaMemcpy(g->inc_dev, g->inc.data(), total * sizeof(unsigned long long),
                               cudaMemcpyHostToDevice));
        YF_CUDA_TRY(cudaMalloc(&g->acc64, (size_t)total * 4 * sizeof(double)));
        YF_CUDA_TRY(cudaMemset(g->acc64, 0, (size_t)total * 4 * sizeof(double)));
        YF_CUDA_TRY(cudaMalloc(&g->acc32, (size_t)total * 4 * sizeof(float)));
        YF_CUDA_TRY(cudaMemset(g->acc32, 0, (size_t)total * 4 * sizeof(float)));
        YF_CUDA_TRY(cudaMalloc(&g->kahan, (size_t)total * 8 * sizeof(float)));
        YF_CUDA_TRY(cudaMemset(g->kahan, 0, (size_t)total * 8 * sizeof(float)));
    }
    if (g->has_src && g->src.kind == YF_WAVE_TABLE && !g->src_table_host.empty()) {
        YF_CUDA_TRY(cudaMalloc(&g->src_table_dev, g->src_table_host.size() * sizeof(double)));
        YF_CUDA_TRY(cudaMemcpy(g->src_table_dev, g->src_table_host.data(),
                               g->src_table_host.size() * sizeof(double), cudaMemcpyHostToDevice));
        g->src_table_len = (long)g->src_table_host.size();
    }
    for (const PortDev &d : g->ports)
        if (g->has_src && d.plane == g->src_plane)
            return fail(YF_E_INVALID, "a port may not sit on the source plane x = %d", d.plane);
    build_segments(g);
    const int nseg = (int)g->segs.size();
    if (nseg > 0) {
        YF_CUDA_TRY(cudaMalloc(&g->segs_dev, nseg * sizeof(EpiSeg)));
        YF_CUDA_TRY(cudaMemcpy(g->segs_dev, g->segs.data(), nseg * sizeof(EpiSeg), cudaMemcpyHostToDevice));
        YF_CUDA_TRY(cudaMalloc(&g->slots, nseg * sizeof(double)));
    }
    // [0] the epilogue's blocks, [1] the source kernel's (the two may run on different streams)
    YF_CUDA_TRY(cudaMalloc(&g->ticket, 2 * sizeof(unsigned int)));
    YF_CUDA_TRY(cudaMemset(g->ticket, 0, 2 * sizeof(unsigned int)));
    if (g->variant >= 2) {
        st = encode_maps(g);
        if (st != YF_OK) return st;
    }
    g->started = true;
    if (g->variant == 2) {
        st = ensure_plan(g);
        if (st != YF_OK) return st;
    }
    if (g->variant == 4) {
        st = enter_tb(g);
        if (st != YF_OK) return st;
    }
    if (g->variant >= 2) YF_CUDA_TRY(side_create(&g->side));
    return YF_OK;
}

template <typename T>
static cudaError_t launch_one_step(yf_grid *g, cudaStream_t s)
{
    cudaError_t e;
    if (g->variant == 4) {
        if ((e = tb_single(g, s)) != cudaSuccess) return e;
    } else if (g->variant >= 1) {
        if (g->variant == 3)
            e = launch_skew<T>(fused_args<T>(g), g->tmF[g->cur], g->tmC, g->tile_y, g->status, s);
        else if (g->variant == 2)
            e = launch_tma_plan<T>(g->plan, g->tile_y, g->cur, g->status, s, &g->side);
        else
            e = launch_fused<T>(fused_args<T>(g), g->tile_y, s);
        if (e != cudaSuccess) return e;
        g->cur ^= 1;
        g->hpar ^= 1;
    } else {
        const StencilParams<T> P = stencil_params<T>(g);
        const Fields<T> F = fields_of<T>(g, g->cur);
        e = launch_update_h<T>(P, F, s);
        if (e != cudaSuccess) return e;
        e = launch_update_e<T>(P, F, s);
        if (e != cudaSuccess) return e;
    }
    return launch_epilogue<T>(epi_params<T>(g), s);
}

// zero fields, CPML auxiliaries, accumulators, counters (geometry and set-up kept)
yf_status reset_state(yf_grid *g)
{
    YF_CUDA_TRY(cudaStreamSynchronize(g->stream));
    for (int b = 0; b < g->nbuf(); ++b) YF_CUDA_TRY(cudaMemsetAsync(g->buf[b], 0, 6 * g->npts * g->esz, g->stream));
    for (int a = 0; a < 3; ++a)
        for (int q = 0; q < 2; ++q) {
            void *ps[3] = {g->psiE[a][q], g->psiH[0][a][q], g->psiH[1][a][q]};
            for (void *p : ps)
                if (p) YF_CUDA_TRY(cudaMemsetAsync(p, 0, g->psi_count[a] * g->esz, g->stream));
        }
    if (g->nf_total > 0) {
        YF_CUDA_TRY(cudaMemsetAsync(g->acc64, 0, (size_t)g->nf_total * 4 * sizeof(double), g->stream));
        YF_CUDA_TRY(cudaMemsetAsync(g->acc32, 0, (size_t)g->nf_total * 4 * sizeof(float), g->stream));
        YF_CUDA_TRY(cudaMemsetAsync(g->kahan, 0, (size_t)g->nf_total * 8 * sizeof(float), g->stream));
    }
    YF_CUDA_TRY(cudaMemsetAsync(g->ctr, 0, 2 * sizeof(long long), g->stream));
    YF_CUDA_TRY(cudaMemsetAsync(g->status, 0, sizeof(int), g->stream));
    g->steps_done = 0;   // the zeroing stays queued: later work on the grid's stream follows it
    return YF_OK;
}

cudaError_t step_direct(yf_grid *g, cudaStream_t s)
{
    return g->prec == YF_FP32 ? launch_one_step<float>(g, s) : launch_one_step<double>(g, s);
}

// graph of one chunk from the current state (buffer, auxiliary copy); the state after a
// chunk equals the state before for variants 1-3 (even chunk) and advances the buffer by
// chunk mod 3 for variant 4, so graphs are kept per state
static int graph_key(const yf_grid *g) { return 2 * g->cur + g->hpar; }

static yf_status capture_chunk(yf_grid *g)
{
    cudaGraph_t graph = nullptr;
    const int key = graph_key(g), c0 = g->cur, h0 = g->hpar;
    tb_unchain(g);
    YF_CUDA_TRY(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    if (g->variant == 4) {
        for (int t = 0; t + 1 < g->chunk && e == cudaSuccess; t += 2) e = tb_pair(g, g->stream);
        if (e == cudaSuccess) e = tb_join(g, g->stream);   // every forked stream rejoins the capture
    } else
        for (int t = 0; t < g->chunk && e == cudaSuccess; ++t) e = step_direct(g, g->stream);
    cudaError_t e2 = cudaStreamEndCapture(g->stream, &graph);
    // capture only records: the state advances when the graph is launched
    g->cur = c0;
    g->hpar = h0;
    tb_unchain(g);
    if (e != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return cuda_fail(e, "capturing step chunk"); }
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&g->graph[key], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { g->graph[key] = nullptr; return cuda_fail(e, "cudaGraphInstantiate"); }
    return YF_OK;
}

// state after one replayed chunk
static void advance_chunk(yf_grid *g)
{
    if (g->variant == 4) {
        g->cur = (g->cur + g->chunk) % 3;   // chunk is even: hpar unchanged
    }
}

}  // namespace yf

using namespace yf;

extern "C" {

const char *yf_last_error(void) { return g_err.c_str(); }

yf_status yf_courant_dt(double dx, double dy, double dz, double courant, double *dt)
{
    if (!dt || !(dx > 0) || !(dy > 0) || !(dz > 0) || !(courant > 0) || courant > 1.0)
        return fail(YF_E_INVALID, "yf_courant_dt: need positive spacings and 0 < courant <= 1");
    *dt = courant * courant_limit_dt(dx, dy, dz);
    return YF_OK;
}

yf_status yf_grid_create(int nx, int ny, int nz, double dx, double dy, double dz, double dt,
                         yf_prec prec, void *stream, yf_grid **out)
{
    if (!out) return fail(YF_E_INVALID, "yf_grid_create: out is NULL");
    *out = nullptr;
    if (nx < 3 || ny < 3 || nz < 3) return fail(YF_E_INVALID, "yf_grid_create: need >= 3 cells per axis");
    if (!(dx > 0) || !(dy > 0) || !(dz > 0)) return fail(YF_E_INVALID, "yf_grid_create: spacings must be > 0");
    if (prec != YF_FP32 && prec != YF_FP64) return fail(YF_E_INVALID, "yf_grid_create: bad precision");
    const double lim = courant_limit_dt(dx, dy, dz);
    if (dt <= 0) dt = 0.99 * lim;
    if (dt > lim * (1.0 + 1e-12))
        return fail(YF_E_UNSTABLE, "dt = %.6g s exceeds the Courant limit %.6g s", dt, lim);
    yf_grid *g = new (std::nothrow) yf_grid();
    if (!g) return fail(YF_E_OOM, "yf_grid_create: host allocation failed");
    g->nx = nx; g->ny = ny; g->nz = nz; g->dx = dx; g->dy = dy; g->dz = dz; g->dt = dt;
    g->prec = prec;
    g->esz = prec == YF_FP32 ? 4 : 8;
    g->px = ((nx + 1) + 31) / 32 * 32;
    g->plane = (long)g->px * (ny + 1);
    g->npts = g->plane * (nz + 1);
    if (stream) {
        g->stream = (cudaStream_t)stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete g; return cuda_fail(e, "cudaStreamCreate"); }
        g->own_stream = true;
    }
    auto bail = [&](cudaError_t e, const char *w) { yf_status s = cuda_fail(e, w); yf_grid_destroy(g); return s; };
    cudaError_t e;
    for (int b = 0; b < 2; ++b) {
        if ((e = cudaMalloc(&g->buf[b], 6 * g->npts * g->esz)) != cudaSuccess) return bail(e, "cudaMalloc fields");
        if ((e = cudaMemset(g->buf[b], 0, 6 * g->npts * g->esz)) != cudaSuccess) return bail(e, "cudaMemset fields");
    }
    g->tile_y = prec == YF_FP32 ? 8 : 8;
    if ((e = cudaMalloc(&g->cls_base, 3 * g->npts)) != cudaSuccess) return bail(e, "cudaMalloc classes");
    if ((e = cudaMemset(g->cls_base, 0, 3 * g->npts)) != cudaSuccess) return bail(e, "cudaMemset classes");
    for (int c = 0; c < 3; ++c) g->cls[c] = g->cls_base + c * g->npts;
    if ((e = cudaMalloc(&g->ctab, 2 * kMaxClasses * g->esz)) != cudaSuccess) return bail(e, "cudaMalloc ctab");
    if ((e = cudaMalloc(&g->eps_tab, kMaxClasses * sizeof(double))) != cudaSuccess) return bail(e, "cudaMalloc eps");
    // [0] steps whose port samples are transformed, [1] steps whose source is added
    if ((e = cudaMalloc(&g->ctr, 2 * sizeof(long long))) != cudaSuccess) return bail(e, "cudaMalloc ctr");
    if ((e = cudaMemset(g->ctr, 0, 2 * sizeof(long long))) != cudaSuccess) return bail(e, "cudaMemset ctr");
    if ((e = cudaMalloc(&g->status, sizeof(int))) != cudaSuccess) return bail(e, "cudaMalloc status");
    if ((e = cudaMemset(g->status, 0, sizeof(int))) != cudaSuccess) return bail(e, "cudaMemset status");
    if ((e = cudaMalloc(&g->energy_partials, (kEnergyBlocks + 1) * sizeof(double))) != cudaSuccess)
        return bail(e, "cudaMalloc energy scratch");
    for (int f = 0; f < 6; ++f) g->bc[f] = YF_BC_PEC;
    *out = g;
    return YF_OK;
}

yf_status yf_grid_destroy(yf_grid *g)
{
    if (!g) return YF_OK;
    if (g->stream) cudaStreamSynchronize(g->stream);
    for (int b = 0; b < 6; ++b)
        if (g->graph[b]) cudaGraphExecDestroy(g->graph[b]);
    tb_free(g);
    for (int b = 0; b < 3; ++b) cudaFree(g->buf[b]);
    cudaFree(g->cls_base);
    for (int a = 0; a < 3; ++a) {
        cudaFree(g->prof[a]);
        for (int q = 0; q < 2; ++q) {
            cudaFree(g->psiE[a][q]);
            cudaFree(g->psiH[0][a][q]);
            cudaFree(g->psiH[1][a][q]);
        }
    }
    cudaFree(g->segs_dev); cudaFree(g->slots); cudaFree(g->ticket);
    free_plan(&g->plan);
    side_destroy(&g->side);
    cudaFree(g->ctab); cudaFree(g->eps_tab); cudaFree(g->ctr); cudaFree(g->status);
    cudaFree(g->energy_partials); cudaFree(g->ports_dev); cudaFree(g->inc_dev);
    cudaFree(g->acc64); cudaFree(g->acc32); cudaFree(g->kahan); cudaFree(g->src_table_dev);
    cudaFree(g->ids_stage);
    mat_scratch_free(&g->mat_scratch);
    if (g->mat_ready) cudaEventDestroy(g->mat_ready);
    if (g->mstream) cudaStreamDestroy(g->mstream);
    if (g->own_stream) cudaStreamDestroy(g->stream);
    delete g;
    return YF_OK;
}

yf_status yf_grid_dt(yf_grid *g, double *dt)
{
    if (!g || !dt) return fail(YF_E_INVALID, "yf_grid_dt: NULL argument");
    *dt = g->dt;
    return YF_OK;
}

yf_status yf_set_materials(yf_grid *g, const uint8_t *ids, yf_mem where, int nmat,
                           const double *eps_r, const double *sigma, const double *mu_r,
                           const uint8_t *is_pec)
{
    if (!g || !ids || !eps_r || !sigma) return fail(YF_E_INVALID, "yf_set_materials: NULL argument");
    if (g->started && !g->geometry_open)
        return fail(YF_E_STATE, "yf_set_materials after the first step (call yf_reset first)");
    if (nmat < 1 || nmat > 256) return fail(YF_E_INVALID, "yf_set_materials: nmat must be 1..256");
    for (int m = 0; m < nmat; ++m) {
        if (!(eps_r[m] > 0) || !(sigma[m] >= 0))
            return fail(YF_E_INVALID, "material %d: need eps_r > 0 and sigma >= 0", m);
        if (mu_r && mu_r[m] != 1.0)
            return fail(YF_E_UNSUPPORTED, "material %d: mu_r != 1 is not supported", m);
    }
    const size_t ncell = (size_t)g->nx * g->ny * g->nz;
    const uint8_t *ids_dev = ids;
    // host ids go through a device staging buffer on the grid's stream; a grid that re-solves
    // after yf_reset keeps that buffer, one set up once (a batch instance) frees it
    const bool keep = g->started;
    cudaStream_t ms = g->stream;
    if (where == YF_HOST) {
        // the copy and the derivation run on the materials stream, beside whatever is queued on
        // the grid's stream (the zeroing of yf_reset); they touch none of its buffers
        if (!g->mstream) YF_CUDA_TRY(cudaStreamCreateWithFlags(&g->mstream, cudaStreamNonBlocking));
        if (!g->mat_ready) YF_CUDA_TRY(cudaEventCreateWithFlags(&g->mat_ready, cudaEventDisableTiming));
        ms = g->mstream;
        if (!g->ids_stage) YF_CUDA_TRY(cudaMalloc(&g->ids_stage, ncell));
        YF_CUDA_TRY(cudaMemcpyAsync(g->ids_stage, ids, ncell, cudaMemcpyHostToDevice, ms));
        ids_dev = g->ids_stage;
    }
    yf_status st = derive_materials(g, ids_dev, nmat, eps_r, sigma, is_pec, ms);
    if (where == YF_HOST) {
        cudaStreamSynchronize(ms);   // the copy has read the caller's ids, also on errors
        // later work on the grid's stream sees the new classes
        cudaError_t e = cudaEventRecord(g->mat_ready, ms);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(g->stream, g->mat_ready, 0);
        if (!keep) {
            cudaFree(g->ids_stage);
            g->ids_stage = nullptr;
        }
        if (st == YF_OK && e != cudaSuccess) return cuda_fail(e, "yf_set_materials: ordering the grid's stream");
    }
    return st;
}

yf_status yf_add_pec_sheet(yf_grid *g, int ax, int index, int lo0, int hi0, int lo1, int hi1)
{
    if (!g) return fail(YF_E_INVALID, "yf_add_pec_sheet: NULL grid");
    if (g->started && !g->geometry_open)
        return fail(YF_E_STATE, "yf_add_pec_sheet after the first step (call yf_reset first)");
    const int N[3] = {g->nx, g->ny, g->nz};
    if (ax < 0 || ax > 2) return fail(YF_E_INVALID, "yf_add_pec_sheet: normal_axis must be 0..2");
    const int a0 = ax == 0 ? 1 : 0, a1 = ax == 2 ? 1 : 2;
    if (index < 0 || index > N[ax] || lo0 < 0 || hi0 > N[a0] || lo0 > hi0 || lo1 < 0 ||
        hi1 > N[a1] || lo1 > hi1)
        return fail(YF_E_INVALID, "yf_add_pec_sheet: rectangle outside the grid");
    const int sh[6] = {ax, index, lo0, hi0, lo1, hi1};
    g->sheets.insert(g->sheets.end(), sh, sh + 6);
    if (g->materials_done) {
        yf_status st = apply_pec_sheet(g->nx, g->ny, g->nz, g->px, g->plane, g->cls, sh, g->stream);
        if (st != YF_OK) return st;
        YF_CUDA_TRY(cudaStreamSynchronize(g->stream));
    }
    return YF_OK;
}

yf_status yf_set_boundaries(yf_grid *g, const int bc[6])
{
    if (!g || !bc) return fail(YF_E_INVALID, "yf_set_boundaries: NULL argument");
    if (g->started) return fail(YF_E_STATE, "yf_set_boundaries after the first step");
    for (int f = 0; f < 6; ++f)
        if (bc[f] != YF_BC_PEC && bc[f] != YF_BC_PML) return fail(YF_E_INVALID, "bad boundary kind");
    for (int f = 0; f < 6; ++f) g->bc[f] = bc[f];
    return YF_OK;
}

yf_status yf_set_pml(yf_grid *g, int ncells, int order, double sigma_scale, double kappa_max,
                     double alpha_max)
{
    if (!g) return fail(YF_E_INVALID, "yf_set_pml: NULL grid");
    if (g->started) return fail(YF_E_STATE, "yf_set_pml after the first step");
    if (ncells < 0 || order < 0 || !(sigma_scale >= 0) || !(kappa_max >= 1) || !(alpha_max >= 0))
        return fail(YF_E_INVALID, "yf_set_pml: bad parameters");
    g->pml_n = ncells; g->pml_order = order; g->pml_sigma_scale = sigma_scale;
    g->pml_kappa_max = kappa_max; g->pml_alpha_max = alpha_max;
    return YF_OK;
}

yf_status yf_set_source(yf_grid *g, int axis, int plane, int j0, int j1, int k0, int k1,
                        const yf_waveform *w)
{
    if (!g || !w) return fail(YF_E_INVALID, "yf_set_source: NULL argument");
    if (g->started) return fail(YF_E_STATE, "yf_set_source after the first step");
    if (axis != 0) return fail(YF_E_UNSUPPORTED, "yf_set_source: only axis 0 (x) is supported");
    if (plane < 1 || plane >= g->nx || j0 < 1 || j1 >= g->ny || j0 > j1 || k0 < 0 || k1 > g->nz ||
        k0 >= k1)
        return fail(YF_E_INVALID, "yf_set_source: rectangle outside the interior E_z edges");
    if (w->kind < YF_WAVE_NONE || w->kind > YF_WAVE_TABLE) return fail(YF_E_INVALID, "bad waveform kind");
    if (w->kind == YF_WAVE_DIFF_GAUSS && !(w->p0 > 0)) return fail(YF_E_INVALID, "sigma must be > 0");
    if (w->kind == YF_WAVE_GAUSS_SINE && !(w->p1 > 0)) return fail(YF_E_INVALID, "bandwidth must be > 0");
    if (w->kind == YF_WAVE_TABLE && (!w->table || w->table_len <= 0))
        return fail(YF_E_INVALID, "table waveform needs a table");
    g->src = *w;
    if (g->src.t0 < 0) {
        if (w->kind == YF_WAVE_DIFF_GAUSS) g->src.t0 = 3.0 * w->p0;
        else if (w->kind == YF_WAVE_GAUSS_SINE) g->src.t0 = 3.0 * (2.0 / (M_PI * w->p1));
        else g->src.t0 = 0.0;
    }
    if (w->kind == YF_WAVE_TABLE) g->src_table_host.assign(w->table, w->table + w->table_len);
    g->src.table = nullptr;
    g->src_plane = plane; g->sj0 = j0; g->sj1 = j1; g->sk0 = k0; g->sk1 = k1;
    g->has_src = w->kind != YF_WAVE_NONE;
    return YF_OK;
}

yf_status yf_add_port(yf_grid *g, const yf_port_desc *d, int nfreq, const double *freqs,
                      int *port_id)
{
    if (!g || !d || !freqs) return fail(YF_E_INVALID, "yf_add_port: NULL argument");
    if (g->started) return fail(YF_E_STATE, "yf_add_port after the first step");
    if ((int)g->ports.size() >= kMaxPorts) return fail(YF_E_UNSUPPORTED, "at most %d ports", kMaxPorts);
    if (d->axis != 0) return fail(YF_E_UNSUPPORTED, "yf_add_port: only axis 0 (x) is supported");
    const int m = d->margin;
    if (d->plane < 1 || d->plane >= g->nx || (d->direction != 1 && d->direction != -1) ||
        d->j0 < 1 || d->j1 >= g->ny || d->j0 >= d->j1 || d->k0 < 0 || d->k1 > g->nz ||
        d->k0 >= d->k1 || m < 1 || d->kb > d->kt || d->j0 - m < 0 || d->j1 + m - 1 > g->ny - 1 ||
        d->kb - m < 0 || d->kt + m - 1 > g->nz - 1)
        return fail(YF_E_INVALID, "yf_add_port: V surface or I loop outside the grid");
    if (nfreq < 1) return fail(YF_E_INVALID, "yf_add_port: nfreq must be >= 1");
    for (int f = 0; f < nfreq; ++f)
        if (!(freqs[f] > 0) || !(freqs[f] * g->dt < 1.0))
            return fail(YF_E_INVALID, "yf_add_port: frequencies must lie in (0, 1/dt)");
    PortDev p;
    p.plane = d->plane; p.dir = d->direction; p.j0 = d->j0; p.j1 = d->j1; p.k0 = d->k0;
    p.k1 = d->k1; p.kb = d->kb; p.kt = d->kt; p.m = m; p.nfreq = nfreq;
    p.foff = (int)g->inc.size();
    const double width = d->width > 0 ? d->width : (d->j1 - d->j0) * g->dy;
    p.vscale = -(g->dy * g->dz) / width;
    for (int f = 0; f < nfreq; ++f) {
        // phase increment per half step as a 64-bit fraction of a turn
        const double x = freqs[f] * g->dt * 0.5;
        g->inc.push_back((unsigned long long)std::llrint(x * 0x1p64));
        g->freqs.push_back(freqs[f]);
    }
    g->ports.push_back(p);
    if (port_id) *port_id = (int)g->ports.size() - 1;
    return YF_OK;
}

yf_status yf_set_dft_mode(yf_grid *g, int mask)
{
    if (!g) return fail(YF_E_INVALID, "yf_set_dft_mode: NULL grid");
    if (g->started) return fail(YF_E_STATE, "yf_set_dft_mode after the first step");
    if (mask <= 0 || (mask & ~(YF_DFT_FP64 | YF_DFT_KAHAN32 | YF_DFT_FP32)))
        return fail(YF_E_INVALID, "yf_set_dft_mode: bad mask");
    g->dft_mask = mask;
    return YF_OK;
}

yf_status yf_step(yf_grid *g, long n)
{
    if (!g) return fail(YF_E_INVALID, "yf_step: NULL grid");
    if (n < 0) return fail(YF_E_INVALID, "yf_step: n < 0");
    yf_status st = finalize(g);
    if (st != YF_OK) return st;
    g->geometry_open = false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    YF_CUDA_TRY(cudaStreamIsCapturing(g->stream, &cs));
    long done = 0;
    if (cs == cudaStreamCaptureStatusNone && n >= g->chunk) {
        for (; done + g->chunk <= n; done += g->chunk) {
            if (!g->graph[graph_key(g)]) {
                st = capture_chunk(g);
                if (st != YF_OK) return st;
            }
            YF_CUDA_TRY(cudaGraphLaunch(g->graph[graph_key(g)], g->stream));
            advance_chunk(g);
        }
    }
    if (g->variant == 4) {
        tb_unchain(g);   // the first direct pair forks after everything queued so far
        for (; done + 2 <= n; done += 2) YF_CUDA_TRY(tb_pair(g, g->stream));
        YF_CUDA_TRY(tb_join(g, g->stream));
        tb_unchain(g);
    }
    for (; done < n; ++done) YF_CUDA_TRY(step_direct(g, g->stream));
    g->steps_done += n;
    return YF_OK;
}

yf_status yf_sync(yf_grid *g)
{
    if (!g) return fail(YF_E_INVALID, "yf_sync: NULL grid");
    YF_CUDA_TRY(cudaStreamSynchronize(g->stream));
    int st = 0;
    YF_CUDA_TRY(cudaMemcpy(&st, g->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st & 4) return fail(YF_E_CUDA, "TMA-staged step: shared memory base not 128-byte aligned");
    if (st & 2) return fail(YF_E_TIMEOUT, "a bounded device wait of the TMA-staged step gave up");
    if (st & 1) return fail(YF_E_UNSTABLE, "a port sample became non-finite");
    return YF_OK;
}

yf_status yf_steps_done(yf_grid *g, long *n)
{
    if (!g || !n) return fail(YF_E_INVALID, "yf_steps_done: NULL argument");
    *n = g->steps_done;
    return YF_OK;
}

yf_status yf_read_fields(yf_grid *g, int comp, void *dst, yf_mem where)
{
    if (!g || !dst || comp < 0 || comp > 5) return fail(YF_E_INVALID, "yf_read_fields: bad argument");
    const size_t w = (size_t)(g->nx + 1) * g->esz;
    YF_CUDA_TRY(cudaMemcpy2DAsync(dst, w, g->fld(comp), (size_t)g->px * g->esz, w,
                                  (size_t)(g->ny + 1) * (g->nz + 1),
                                  where == YF_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                  g->stream));
    YF_CUDA_TRY(cudaStreamSynchronize(g->stream));
    return YF_OK;
}

yf_status yf_write_fields(yf_grid *g, int comp, const void *src, yf_mem where)
{
    if (!g || !src || comp < 0 || comp > 5) return fail(YF_E_INVALID, "yf_write_fields: bad argument");
    if (!g->materials_done) {
        // classes decide which edges are PEC; settle the default materials first
        uint8_t *ids = nullptr;
        const size_t ncell = (size_t)g->nx * g->ny * g->nz;
        YF_CUDA_TRY(cudaMalloc(&ids, ncell));
        YF_CUDA_TRY(cudaMemset(ids, 0, ncell));
        const double er = 1.0, sg = 0.0;
        const uint8_t pec = 0;
        yf_status st = derive_materials(g, ids, 1, &er, &sg, &pec, g->stream);
        cudaFree(ids);
        if (st != YF_OK) return st;
    }
    const size_t w = (size_t)(g->nx + 1) * g->esz;
    YF_CUDA_TRY(cudaMemcpy2DAsync(g->fld(comp), (size_t)g->px * g->esz, src, w, w,
                                  (size_t)(g->ny + 1) * (g->nz + 1),
                                  where == YF_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                  g->stream));
    cudaError_t e;
    if (g->prec == YF_FP32)
        e = launch_sanitize<float>(fields_of<float>(g, g->cur), g->cls, g->nx, g->ny, g->nz, g->px,
                                   g->plane, g->stream);
    else
        e = launch_sanitize<double>(fields_of<double>(g, g->cur), g->cls, g->nx, g->ny, g->nz, g->px,
                                    g->plane, g->stream);
    YF_CUDA_TRY(e);
    // every field buffer carries the written component: the TMA-staged step skips the node
    // column i = nx and row j = ny when they form a tile of their own, and there the two
    // buffers must already agree (only H_x at i = nx and H_y at j = ny live there, and the
    // update leaves them unchanged: their tangential E neighbours are PEC)
    const size_t bytes = (size_t)g->npts * g->esz;
    for (int b = 0; b < g->nbuf(); ++b)
        if (b != g->cur)
            YF_CUDA_TRY(cudaMemcpyAsync((char *)g->buf[b] + (size_t)comp * bytes, g->fld(comp), bytes,
                                        cudaMemcpyDeviceToDevice, g->stream));
    YF_CUDA_TRY(cudaStreamSynchronize(g->stream));
    return YF_OK;
}

yf_status yf_energy(yf_grid *g, double *w)
{
    if (!g || !w) return fail(YF_E_INVALID, "yf_energy: NULL argument");
    if (!g->materials_done) { *w = 0.0; }
    double *out = g->energy_partials + kEnergyBlocks;
    cudaError_t e;
    if (g->prec == YF_FP32) {
        const float *c[6];
        for (int q = 0; q < 6; ++q) c[q] = (const float *)g->fld(q);
        e = launch_energy<float>(c, g->cls, g->eps_tab, g->nx, g->ny, g->nz, g->px, g->plane,
                                 g->energy_partials, out, g->stream);
    } else {
        const double *c[6];
        for (int q = 0; q < 6; ++q) c[q] = (const double *)g->fld(q);
        e = launch_energy<double>(c, g->cls, g->eps_tab, g->nx, g->ny, g->nz, g->px, g->plane,
                                  g->energy_partials, out, g->stream);
    }
    YF_CUDA_TRY(e);
    double r = 0.0;
    YF_CUDA_TRY(cudaMemcpyAsync(&r, out, sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    YF_CUDA_TRY(cudaStreamSynchronize(g->stream));
    *w = r * g->dx * g->dy * g->dz;
    return YF_OK;
}

yf_status yf_read_port_dft(yf_grid *g, int port, int kind, double *V_re, double *V_im,
                           double *I_re, double *I_im)
{
    if (!g || port < 0 || port >= (int)g->ports.size())
        return fail(YF_E_INVALID, "yf_read_port_dft: bad port");
    if (kind != YF_DFT_FP64 && kind != YF_DFT_KAHAN32 && kind != YF_DFT_FP32)
        return fail(YF_E_INVALID, "yf_read_port_dft: bad accumulator kind");
    const PortDev &p = g->ports[port];
    const int nf = p.nfreq;
    std::vector<double> v(4 * (size_t)nf, 0.0);
    if (g->started) {
        if (!(g->dft_mask & kind)) return fail(YF_E_STATE, "accumulator kind was not enabled");
        YF_CUDA_TRY(cudaStreamSynchronize(g->stream));
        if (kind == YF_DFT_FP64) {
            YF_CUDA_TRY(cudaMemcpy(v.data(), g->acc64 + 4 * (size_t)p.foff, 4 * nf * sizeof(double),
                                   cudaMemcpyDeviceToHost));
        } else if (kind == YF_DFT_FP32) {
            std::vector<float> f(4 * (size_t)nf);
            YF_CUDA_TRY(cudaMemcpy(f.data(), g->acc32 + 4 * (size_t)p.foff, 4 * nf * sizeof(float),
                                   cudaMemcpyDeviceToHost));
            for (size_t q = 0; q < f.size(); ++q) v[q] = f[q];
        } else {
            std::vector<float> f(8 * (size_t)nf);
            YF_CUDA_TRY(cudaMemcpy(f.data(), g->kahan + 8 * (size_t)p.foff, 8 * nf * sizeof(float),
                                   cudaMemcpyDeviceToHost));
            for (size_t q = 0; q < 4 * (size_t)nf; ++q) v[q] = (double)f[2 * q] - (double)f[2 * q + 1];
        }
    }
    for (int f = 0; f < nf; ++f) {
        if (V_re) V_re[f] = v[4 * f + 0] * g->dt;
        if (V_im) V_im[f] = v[4 * f + 1] * g->dt;
        if (I_re) I_re[f] = v[4 * f + 2] * g->dt;
        if (I_im) I_im[f] = v[4 * f + 3] * g->dt;
    }
    return YF_OK;
}

yf_status yf_read_sparams_acc(yf_grid *g, int kind, double z_ref, double *S_star, double *S,
                              double *Zr, double *Zc, double *tau)
{
    if (!g) return fail(YF_E_INVALID, "yf_read_sparams: NULL grid");
    if (g->ports.size() != 2) return fail(YF_E_INVALID, "yf_read_sparams: needs exactly two ports");
    const int nf = g->ports[0].nfreq;
    if (g->ports[1].nfreq != nf) return fail(YF_E_INVALID, "yf_read_sparams: ports differ in frequencies");
    for (int f = 0; f < nf; ++f)
        if (g->freqs[f] != g->freqs[nf + f])
            return fail(YF_E_INVALID, "yf_read_sparams: ports differ in frequencies");
    std::vector<double> d(8 * (size_t)nf);
    for (int p = 0; p < 2; ++p) {
        yf_status st = yf_read_port_dft(g, p, kind, &d[(4 * p + 0) * nf], &d[(4 * p + 1) * nf],
                                        &d[(4 * p + 2) * nf], &d[(4 * p + 3) * nf]);
        if (st != YF_OK) return st;
    }
    return sparams_uniform(nf, g->freqs.data(), d.data(), g->ports[1].dir, z_ref, S_star, S, Zr, Zc, tau);
}

yf_status yf_read_sparams(yf_grid *g, double z_ref, double *S_star, double *S, double *Zr,
                          double *Zc, double *tau)
{
    return yf_read_sparams_acc(g, YF_DFT_FP64, z_ref, S_star, S, Zr, Zc, tau);
}

yf_status yf_reset(yf_grid *g)
{
    if (!g) return fail(YF_E_INVALID, "yf_reset: NULL grid");
    yf_status st = reset_state(g);
    if (st != YF_OK) return st;
    g->sheets.clear();
    g->geometry_open = true;
    return YF_OK;
}

}  // extern "C"

template <typename T>
static cudaError_t profile_one(yf_grid *g, cudaEvent_t *ev, int *nk)
{
    cudaError_t e;
    cudaEventRecord(ev[0], g->stream);
    if (g->variant >= 1) {
        if (g->variant == 3)
            e = launch_skew<T>(fused_args<T>(g), g->tmF[g->cur], g->tmC, g->tile_y, g->status, g->stream);
        else if (g->variant == 2)
            e = launch_tma_plan<T>(g->plan, g->tile_y, g->cur, g->status, g->stream, &g->side);
        else
            e = launch_fused<T>(fused_args<T>(g), g->tile_y, g->stream);
        if (e != cudaSuccess) return e;
        g->cur ^= 1;
        g->hpar ^= 1;
        cudaEventRecord(ev[1], g->stream);
        *nk = 2;
    } else {
        const StencilParams<T> P = stencil_params<T>(g);
        const Fields<T> F = fields_of<T>(g, g->cur);
        if ((e = launch_update_h<T>(P, F, g->stream)) != cudaSuccess) return e;
        cudaEventRecord(ev[1], g->stream);
        if ((e = launch_update_e<T>(P, F, g->stream)) != cudaSuccess) return e;
        cudaEventRecord(ev[2], g->stream);
        *nk = 3;
    }
    e = launch_epilogue<T>(epi_params<T>(g), g->stream);
    cudaEventRecord(ev[*nk], g->stream);
    return e;
}

// variant 4: pairs of steps; per launch the box kernel (one per pair), the first frame step
// (beside the box kernel), the second frame step (after it), the source (two per pair, on the
// critical path) and the port integrals with the transforms (two per pair, side stream)
static yf_status profile_tb(yf_grid *g, long n, double *ms, int *nkern)
{
    cudaEvent_t ev[12];
    for (int q = 0; q < 12; ++q) YF_CUDA_TRY(cudaEventCreate(&ev[q]));
    const long pairs = n < 2 ? 1 : n / 2;
    double acc[5] = {0, 0, 0, 0, 0};
    cudaError_t e = cudaSuccess;
    for (long t = 0; t < pairs && e == cudaSuccess; ++t) {
        tb_unchain(g);   // each traced pair on its own
        e = tb_pair(g, g->stream, ev);
        if (e == cudaSuccess) e = tb_join(g, g->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
        float m[7] = {0, 0, 0, 0, 0, 0, 0};
        const int from[7] = {0, 2, 3, 5, 6, 8, 10}, to[7] = {1, 3, 4, 6, 7, 9, 11};
        for (int q = 0; q < 7 && e == cudaSuccess; ++q) e = cudaEventElapsedTime(&m[q], ev[from[q]], ev[to[q]]);
        acc[0] += m[0];
        acc[1] += m[1];
        acc[2] += m[3];
        acc[3] += 0.5 * (m[2] + m[4]);
        acc[4] += 0.5 * (m[5] + m[6]);
    }
    tb_unchain(g);
    for (int q = 0; q < 12; ++q) cudaEventDestroy(ev[q]);
    YF_CUDA_TRY(e);
    g->steps_done += 2 * pairs;
    for (int q = 0; q < 5; ++q) ms[q] = acc[q] / (double)pairs;
    *nkern = 5;
    return YF_OK;
}

extern "C" yf_status yf_profile_steps(yf_grid *g, long n, double *ms, int *nkern)
{
    if (!g || !ms || !nkern || n < 1) return fail(YF_E_INVALID, "yf_profile_steps: bad argument");
    yf_status st = finalize(g);
    if (st != YF_OK) return st;
    if (g->variant == 4) return profile_tb(g, n, ms, nkern);
    cudaEvent_t ev[4];
    for (int q = 0; q < 4; ++q) YF_CUDA_TRY(cudaEventCreate(&ev[q]));
    double acc[3] = {0, 0, 0};
    int nk = 0;
    cudaError_t e = cudaSuccess;
    for (long t = 0; t < n && e == cudaSuccess; ++t) {
        e = g->prec == YF_FP32 ? profile_one<float>(g, ev, &nk) : profile_one<double>(g, ev, &nk);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[nk]);
        for (int q = 0; q < nk && e == cudaSuccess; ++q) {
            float m = 0.f;
            e = cudaEventElapsedTime(&m, ev[q], ev[q + 1]);
            acc[q] += m;
        }
    }
    for (int q = 0; q < 4; ++q) cudaEventDestroy(ev[q]);
    YF_CUDA_TRY(e);
    g->steps_done += n;
    for (int q = 0; q < nk; ++q) ms[q] = acc[q] / (double)n;
    *nkern = nk;
    return YF_OK;
}

extern "C" {

const char *yf_kernel_name(yf_grid *g, int idx)
{
    static const char *ref[] = {"k_update_h", "k_update_e", "k_epilogue"};
    static const char *fused[] = {"k_yee_fused", "k_epilogue"};
    static const char *tma[] = {"k_yee_tma_batch", "k_epilogue"};
    static const char *skew[] = {"k_yee_skew", "k_epilogue"};
    static const char *tb[] = {"k_yee_tb2", "k_yee_tma_batch (frame step 1)", "k_yee_tma_batch (frame step 2)",
                               "k_epi_source", "k_epilogue (ports and transforms, side stream)"};
    if (!g) return "";
    if (g->variant == 4) return (idx >= 0 && idx < 5) ? tb[idx] : "";
    if (g->variant == 3) return (idx >= 0 && idx < 2) ? skew[idx] : "";
    if (g->variant == 1) return (idx >= 0 && idx < 2) ? fused[idx] : "";
    if (g->variant == 2) return (idx >= 0 && idx < 2) ? tma[idx] : "";
    return (idx >= 0 && idx < 3) ? ref[idx] : "";
}

yf_status yf_launches_per_step(yf_grid *g, int *n)
{
    if (!g || !n) return fail(YF_E_INVALID, "yf_launches_per_step: NULL argument");
    yf_status st = finalize(g);
    if (st != YF_OK) return st;
    if (g->variant == 4) {
        *n = (tb_launches_pair(g) + 1) / 2;
        return YF_OK;
    }
    int k = 0;
    if (g->variant == 0) k = 2;
    else if (g->variant == 2)
        for (int q = 0; q < 5; ++q) k += g->plan.count[q] > 0;
    else k = 1;
    *n = k + 1;
    return YF_OK;
}

yf_status yf_launches(yf_grid *g, long nsteps, long *n)
{
    if (!g || !n || nsteps < 0) return fail(YF_E_INVALID, "yf_launches: bad argument");
    yf_status st = finalize(g);
    if (st != YF_OK) return st;
    if (g->variant == 4) {
        *n = (nsteps / 2) * tb_launches_pair(g) + (nsteps % 2) * tb_launches_single(g);
        return YF_OK;
    }
    int k = 0;
    st = yf_launches_per_step(g, &k);
    if (st != YF_OK) return st;
    *n = nsteps * k;
    return YF_OK;
}

yf_status yf_tb_box(yf_grid *g, int box[6])
{
    if (!g || !box) return fail(YF_E_INVALID, "yf_tb_box: NULL argument");
    if (g->variant != 4) return fail(YF_E_STATE, "yf_tb_box: variant 4 is not set");
    yf_status st = finalize(g);
    if (st != YF_OK) return st;
    for (int q = 0; q < 6; ++q) box[q] = g->tb->count > 0 ? g->tb->box[q] : -1;
    return YF_OK;
}

yf_status yf_set_variant(yf_grid *g, int variant, int tile_y, int kseg)
{
    if (!g) return fail(YF_E_INVALID, "yf_set_variant: NULL grid");
    if (variant < 0 || variant > 4) return fail(YF_E_INVALID, "yf_set_variant: variant must be 0..4");
    if (variant == 4 && g->prec != YF_FP32) return fail(YF_E_INVALID, "yf_set_variant: variant 4 needs FP32 fields");
    if (tile_y != 4 && tile_y != 8 && tile_y != 16) return fail(YF_E_INVALID, "yf_set_variant: tile_y must be 4, 8 or 16");
    if (kseg < 1 || kseg > kMaxKseg) return fail(YF_E_INVALID, "yf_set_variant: kseg must be 1..%d", kMaxKseg);
    YF_CUDA_TRY(cudaStreamSynchronize(g->stream));
    for (int b = 0; b < 6; ++b)
        if (g->graph[b]) { cudaGraphExecDestroy(g->graph[b]); g->graph[b] = nullptr; }
    if (g->tb || g->buf[2]) {
        yf_status st = leave_tb(g);
        if (st != YF_OK) return st;
    }
    g->variant = variant;
    g->tile_y = tile_y;
    g->kseg = kseg;
    if (g->plan_ok) {
        free_plan(&g->plan);
        g->plan_ok = false;
    }
    if (g->started && variant >= 2) {
        yf_status st = encode_maps(g);
        if (st != YF_OK) return st;
    }
    if (g->started && variant == 2) {
        yf_status st = ensure_plan(g);
        if (st != YF_OK) return st;
    }
    if (g->started && variant == 4) {
        yf_status st = enter_tb(g);
        if (st != YF_OK) return st;
    }
    if (g->started && variant >= 2) YF_CUDA_TRY(side_create(&g->side));
    return YF_OK;
}

yf_status yf_set_box_shape(yf_grid *g, int tile_y, int planes)
{
    if (!g) return fail(YF_E_INVALID, "yf_set_box_shape: NULL grid");
    if (tile_y != 0 && tile_y != 8 && tile_y != 16)
        return fail(YF_E_INVALID, "yf_set_box_shape: tile_y must be 0, 8 or 16");
    if (planes < 0) return fail(YF_E_INVALID, "yf_set_box_shape: planes must be >= 0");
    YF_CUDA_TRY(cudaStreamSynchronize(g->stream));
    for (int b = 0; b < 6; ++b)
        if (g->graph[b]) { cudaGraphExecDestroy(g->graph[b]); g->graph[b] = nullptr; }
    const bool had_tb = g->tb != nullptr;
    if (had_tb) tb_free(g);
    g->box_ty = tile_y == 0 ? 8 : tile_y;
    g->box_seg = planes;
    if (had_tb) return tb_build(g);
    return YF_OK;
}

// checkpoint: header, fields, CPML auxiliaries, accumulators, counters
struct CkptHeader {
    char magic[8];
    int nx, ny, nz, prec, pml_n, nf_total;
    long steps;
    long long ctr;
    int status;
};

yf_status yf_checkpoint_save(yf_grid *g, const char *path)
{
    if (!g || !path) return fail(YF_E_INVALID, "yf_checkpoint_save: NULL argument");
    yf_status st = finalize(g);
    if (st != YF_OK) return st;
    YF_CUDA_TRY(cudaStreamSynchronize(g->stream));
    FILE *fp = fopen(path, "wb");
    if (!fp) return fail(YF_E_INVALID, "cannot open %s for writing", path);
    CkptHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, "YFCKPT1", 8);
    h.nx = g->nx; h.ny = g->ny; h.nz = g->nz; h.prec = g->prec; h.pml_n = g->pml_n;
    h.nf_total = g->nf_total; h.steps = g->steps_done;
    cudaMemcpy(&h.ctr, g->ctr, sizeof(long long), cudaMemcpyDeviceToHost);
    cudaMemcpy(&h.status, g->status, sizeof(int), cudaMemcpyDeviceToHost);
    bool ok = fwrite(&h, sizeof(h), 1, fp) == 1;
    auto dump = [&](const void *dev, size_t bytes) {
        if (!ok || !dev || bytes == 0) return;
        std::vector<char> buf(bytes);
        ok = cudaMemcpy(buf.data(), dev, bytes, cudaMemcpyDeviceToHost) == cudaSuccess &&
             fwrite(buf.data(), 1, bytes, fp) == bytes;
    };
    dump(g->buf[g->cur], 6 * g->npts * g->esz);
    for (int a = 0; a < 3; ++a)
        for (int q = 0; q < 2; ++q) {
            dump(g->psiE[a][q], g->psi_count[a] * g->esz);
            dump(g->psiH[g->hpar][a][q], g->psi_count[a] * g->esz);
        }
    dump(g->acc64, (size_t)g->nf_total * 4 * sizeof(double));
    dump(g->acc32, (size_t)g->nf_total * 4 * sizeof(float));
    dump(g->kahan, (size_t)g->nf_total * 8 * sizeof(float));
    fclose(fp);
    if (!ok) return fail(YF_E_CUDA, "checkpoint write to %s failed", path);
    return YF_OK;
}

yf_status yf_checkpoint_load(yf_grid *g, const char *path)
{
    if (!g || !path) return fail(YF_E_INVALID, "yf_checkpoint_load: NULL argument");
    yf_status st = finalize(g);
    if (st != YF_OK) return st;
    YF_CUDA_TRY(cudaStreamSynchronize(g->stream));
    FILE *fp = fopen(path, "rb");
    if (!fp) return fail(YF_E_INVALID, "cannot open %s", path);
    CkptHeader h;
    if (fread(&h, sizeof(h), 1, fp) != 1 || memcmp(h.magic, "YFCKPT1", 8) != 0 || h.nx != g->nx ||
        h.ny != g->ny || h.nz != g->nz || h.prec != g->prec || h.pml_n != g->pml_n ||
        h.nf_total != g->nf_total) {
        fclose(fp);
        return fail(YF_E_INVALID, "checkpoint %s does not match this grid", path);
    }
    bool ok = true;
    auto load = [&](void *dev, size_t bytes) {
        if (!ok || !dev || bytes == 0) return;
        std::vector<char> buf(bytes);
        ok = fread(buf.data(), 1, bytes, fp) == bytes &&
             cudaMemcpy(dev, buf.data(), bytes, cudaMemcpyHostToDevice) == cudaSuccess;
    };
    load(g->buf[g->cur], 6 * g->npts * g->esz);
    for (int a = 0; a < 3; ++a)
        for (int q = 0; q < 2; ++q) {
            load(g->psiE[a][q], g->psi_count[a] * g->esz);
            load(g->psiH[g->hpar][a][q], g->psi_count[a] * g->esz);
        }
    load(g->acc64, (size_t)g->nf_total * 4 * sizeof(double));
    load(g->acc32, (size_t)g->nf_total * 4 * sizeof(float));
    load(g->kahan, (size_t)g->nf_total * 8 * sizeof(float));
    fclose(fp);
    if (!ok) return fail(YF_E_INVALID, "checkpoint %s is truncated", path);
    // the other field buffers must agree on the nodes a step leaves untouched
    for (int b = 0; b < g->nbuf(); ++b)
        if (b != g->cur)
            YF_CUDA_TRY(cudaMemcpy(g->buf[b], g->buf[g->cur], 6 * g->npts * g->esz, cudaMemcpyDeviceToDevice));
    YF_CUDA_TRY(cudaMemcpy(g->ctr, &h.ctr, sizeof(long long), cudaMemcpyHostToDevice));
    YF_CUDA_TRY(cudaMemcpy(g->ctr + 1, &h.ctr, sizeof(long long), cudaMemcpyHostToDevice));
    YF_CUDA_TRY(cudaMemcpy(g->status, &h.status, sizeof(int), cudaMemcpyHostToDevice));
    g->steps_done = h.steps;
    return YF_OK;
}

}  // extern "C"
